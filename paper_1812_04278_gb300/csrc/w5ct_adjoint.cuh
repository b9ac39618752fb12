// w5ct_adjoint.cuh -- adjoint (vector-Jacobian product) of one RK4 + CT step
// of fixed dt, and of the initial-condition map from primitive fields and an
// edge vector potential.
//
// One step is linear in its stage results: with D_s the flux divergence and
// Omega_s the corner EMFs of stage s (Sec. 2.1, Eq. num, Eqs. ox1-ox3),
//   q_{s+1} = q^n + c_s dt D_s,   b_{s+1} = b^n + c_s dt curl Omega_s  (s < 3),
//   q^{n+1} = q^n + dt sum_s w_s D_s,   b^{n+1} = b^n + dt curl sum_s w_s Omega_s,
// c = (1/2, 1/2, 1), w = (1, 2, 2, 1)/6.  (D_s, Omega_s) depend on the stage
// state through the sweeps (nonlinear, per face) and the divergence, EMF
// average and cell-field interpolation (linear).  The adjoint runs the
// stages backwards: the linear maps by their transposes (the kernels below),
// the sweeps by adj_face_kernel, the reverse mode of each face's function
// (48 inputs -> 7 outputs) contracted with the incoming flux adjoints.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "w5ct_kernels.cuh"

namespace w5ct {

// ---------------------------------------------------------------- sweep adjoint

template <typename B>
struct AdjSweepArgs {
    int nx, ny, nz;
    const B *q[5];          // stage state (rho, m, E), arithmetic type
    const B *bc[3];         // the stage's cell-centred field
    const double *lamF[5];  // dL/dF of this axis' face fluxes (lab order)
    const double *lamS[2];  // dL/dS of this axis' transport fluxes
    double *cb;             // 48 planes: cb[(s * 8 + v) * n + p] = d(lam . out_p)/d(input v of stencil cell s)
    Phys<B> K;
};

// ---------------------------------------------------------------- reverse mode

// The seven characteristic modes of Appendix A at the interface state w =
// (rho, v_n, v_t1, v_t2, B_n, B_t1, B_t2, P) as full left and right
// eigenvectors in the frame order (rho, m_n, m_t1, m_t2, B_t1, B_t2, E):
// modes 0/1 fast (v -/+ c_f), 2/3 slow (v -/+ c_slow), 4/5 Alfven
// (v -/+ c_A), 6 entropy.  The formulas (and branches) of face_flux, written
// as whole vectors: the paired forms there are L = Lc +- Ls, R = Rc +- Rs.
template <typename Real>
__device__ __forceinline__ void eigen7(const Real (&w)[8], const Phys<Real> &K, Real (&L)[7][7], Real (&R)[7][7]) {
    using m = M<Real>;
    const Real r = w[0], vn = w[1], vt1 = w[2], vt2 = w[3], Bn = w[4], Bt1 = w[5], Bt2 = w[6], P = w[7];
    const Real ir = m::rcp_(r);
    const Real ca2 = Bn * Bn * ir;
    const Real btm = Bt1 * Bt1 + Bt2 * Bt2;
    const Real bt2 = btm * ir;
    const Real v2 = vn * vn + vt1 * vt1 + vt2 * vt2;
    Real cs2 = K.gamma * P * ir;
    if constexpr (float_based<Real>) cs2 = m::max_(cs2, K.cs2_rel * (v2 + ca2 + bt2));
    Real fmc, cms, cf2, csl2;
    speeds<Real>(cs2, ca2, bt2, fmc, cms, cf2, csl2);
    const Real cf = m::sqrt_(cf2), csl = m::sqrt_(csl2), cs = m::sqrt_(cs2);
    const Real dfs = fmc + cms;
    Real af, as;
    if (dfs >= K.eps_b2) {
        const Real idf = m::rcp_(dfs);
        af = m::sqrt_(m::max_(cms * idf, Real(0)));
        as = m::sqrt_(m::max_(fmc * idf, Real(0)));
    } else {
        af = Real(1);
        as = Real(1);
    }
    Real b1, b2;
    if (btm > K.eps_b) {
        const Real ib = m::rsqrt_(btm);
        b1 = Bt1 * ib;
        b2 = Bt2 * ib;
    } else {
        b1 = Real(0.70710678118654752440);
        b2 = Real(0.70710678118654752440);
    }
    const Real sg = (Bn >= K.eps_b) ? Real(1) : Real(-1);
    const Real sr = m::sqrt_(r);
    const Real isr = sr * ir;
    const Real bv = b1 * vt1 + b2 * vt2;
    const Real Gf = af * cf * vn - as * csl * sg * bv;
    const Real Ga = sg * (b2 * vt1 - b1 * vt2);
    const Real Gs = as * csl * vn + af * cf * sg * bv;
    const Real ics2 = m::rcp_(cs2);
    const Real pre = Real(0.5) * ics2;
    const Real tau = K.gm1 * ics2;
    auto pair = [&](int mu, const Real (&Lc)[7], const Real (&Ls)[4], const Real (&Rc)[7], const Real (&Rs)[4]) {
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            L[mu][c] = Lc[c];
            L[mu + 1][c] = Lc[c];
            R[mu][c] = Rc[c];
            R[mu + 1][c] = Rc[c];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            L[mu][c] = L[mu][c] + Ls[c];
            L[mu + 1][c] = L[mu + 1][c] - Ls[c];
        }
        const int rows[4] = {1, 2, 3, 6};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            R[mu][rows[k]] = R[mu][rows[k]] + Rs[k];
            R[mu + 1][rows[k]] = R[mu + 1][rows[k]] - Rs[k];
        }
    };
    {
        const Real k1 = -K.gm1 * af;
        const Real Lc[7] = {pre * K.g1 * af * v2, pre * k1 * vn, pre * k1 * vt1, pre * k1 * vt2,
                            pre * (k1 * Bt1 + sr * cs * as * b1), pre * (k1 * Bt2 + sr * cs * as * b2), pre * K.gm1 * af};
        const Real Ls[4] = {pre * Gf, -pre * af * cf, pre * csl * as * b1 * sg, pre * csl * as * b2 * sg};
        const Real Rc[7] = {af, af * vn, af * vt1, af * vt2, cs * as * b1 * isr, cs * as * b2 * isr,
                            af * (Real(0.5) * v2 + cf2 - K.g2 * cs2)};
        const Real Rs[4] = {-af * cf, csl * as * b1 * sg, csl * as * b2 * sg, -Gf};
        pair(0, Lc, Ls, Rc, Rs);
    }
    {
        const Real k2 = -K.gm1 * as;
        const Real Lc[7] = {pre * K.g1 * as * v2, pre * k2 * vn, pre * k2 * vt1, pre * k2 * vt2,
                            pre * (k2 * Bt1 - sr * cs * af * b1), pre * (k2 * Bt2 - sr * cs * af * b2), pre * K.gm1 * as};
        const Real Ls[4] = {pre * Gs, -pre * as * csl, -pre * cf * af * b1 * sg, -pre * cf * af * b2 * sg};
        const Real Rc[7] = {as, as * vn, as * vt1, as * vt2, -cs * af * b1 * isr, -cs * af * b2 * isr,
                            as * (Real(0.5) * v2 + csl2 - K.g2 * cs2)};
        const Real Rs[4] = {-as * csl, -cf * af * b1 * sg, -cf * af * b2 * sg, -Gs};
        pair(2, Lc, Ls, Rc, Rs);
    }
    {
        const Real l0 = Real(0.5) * Ga, l2 = Real(-0.5) * b2 * sg, l3 = Real(0.5) * b1 * sg;
        const Real l4 = Real(-0.5) * sr * b2, l5 = Real(0.5) * sr * b1;
        const Real z = Real(0);
        const Real La[7] = {l0, z, l2, l3, l4, l5, z}, Lb[7] = {l0, z, l2, l3, -l4, -l5, z};
        const Real Ra[7] = {z, z, -b2 * sg, b1 * sg, -b2 * isr, b1 * isr, -Ga};
        const Real Rb[7] = {z, z, -b2 * sg, b1 * sg, b2 * isr, -b1 * isr, -Ga};
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            L[4][c] = La[c];
            L[5][c] = Lb[c];
            R[4][c] = Ra[c];
            R[5][c] = Rb[c];
        }
    }
    {
        const Real Le[7] = {Real(1) - Real(0.5) * tau * v2, tau * vn, tau * vt1, tau * vt2, tau * Bt1, tau * Bt2, -tau};
        const Real Re[7] = {Real(1), vn, vt1, vt2, Real(0), Real(0), Real(0.5) * v2};
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            L[6][c] = Le[c];
            R[6][c] = Re[c];
        }
    }
}

// Reverse of speeds(): adds to (lcs2, lca2, lbt2) the adjoints of its inputs
// given those of (fmc, cms, cf2, csl2); the same branches and guards as the
// forward formulas (Eqs. slow/fast), run backwards.
template <typename B, typename A>
__device__ __forceinline__ void speeds_rev(B cs2, B ca2, B bt2, A lfmc, A lcms, A lcf2, A lcsl2, A &lcs2, A &lca2,
                                           A &lbt2) {
    using m = M<B>;
    const B dd = (cs2 - ca2) * (cs2 - ca2) + bt2 * (bt2 + B(2) * ca2 + B(2) * cs2);
    const B sd = m::sqrt_(dd);
    const B aa = ca2 + bt2 - cs2;
    B fmc, cms;
    if (aa >= B(0)) {
        fmc = B(0.5) * (aa + sd);
        cms = fmc > B(0) ? m::div_(cs2 * bt2, fmc) : B(0);
    } else {
        cms = B(0.5) * (sd - aa);
        fmc = cms > B(0) ? m::div_(cs2 * bt2, cms) : B(0);
    }
    const B cf2 = cs2 + fmc;
    if (cf2 > B(0)) {
        const A icf = A(1) / (A)cf2;
        const A csl2 = (A)m::div_(cs2 * ca2, cf2);
        lcs2 += lcsl2 * (A)ca2 * icf;
        lca2 += lcsl2 * (A)cs2 * icf;
        lcf2 -= lcsl2 * csl2 * icf;
    }
    lcs2 += lcf2;
    lfmc += lcf2;
    A laa = A(0), lsd = A(0);
    if (aa >= B(0)) {
        if (fmc > B(0)) {
            const A ifm = A(1) / (A)fmc;
            lcs2 += lcms * (A)bt2 * ifm;
            lbt2 += lcms * (A)cs2 * ifm;
            lfmc -= lcms * (A)cms * ifm;
        }
        laa += A(0.5) * lfmc;
        lsd += A(0.5) * lfmc;
    } else {
        if (cms > B(0)) {
            const A icm = A(1) / (A)cms;
            lcs2 += lfmc * (A)bt2 * icm;
            lbt2 += lfmc * (A)cs2 * icm;
            lcms -= lfmc * (A)fmc * icm;
        }
        lsd += A(0.5) * lcms;
        laa -= A(0.5) * lcms;
    }
    lca2 += laa;
    lbt2 += laa;
    lcs2 -= laa;
    const A ldd = sd > B(0) ? lsd * A(0.5) / (A)sd : A(0);
    lcs2 += ldd * (A(2) * ((A)cs2 - (A)ca2) + A(2) * (A)bt2);
    lca2 += ldd * (A(-2) * ((A)cs2 - (A)ca2) + A(2) * (A)bt2);
    lbt2 += ldd * (A(2) * (A)bt2 + A(2) * (A)ca2 + A(2) * (A)cs2);
}

// Reverse of eigen7: lw = d/dw of sum(lL * L) + sum(lR * R) at the
// interface state w, written by hand from the forward formulas (recomputed
// here in B; the adjoints in A).  Branches follow the primal values: the
// epsilon_B switches and the WENO sign sg, the c_s^2 bound of the float
// path, the sqrt of zero (subgradient 0): the derivative of the branch the
// forward step takes.
template <typename B, typename A>
__device__ __forceinline__ void eigen7_rev(const B (&w)[8], const Phys<B> &K, const A (&lL)[7][7], const A (&lR)[7][7],
                                           A (&lw)[8]) {
    using m = M<B>;
    const B r = w[0], vn = w[1], vt1 = w[2], vt2 = w[3], Bn = w[4], Bt1 = w[5], Bt2 = w[6], P = w[7];
    // ---- forward values
    const B ir = m::rcp_(r);
    const B ca2 = Bn * Bn * ir;
    const B btm = Bt1 * Bt1 + Bt2 * Bt2;
    const B bt2 = btm * ir;
    const B v2 = vn * vn + vt1 * vt1 + vt2 * vt2;
    const B cs2a = K.gamma * P * ir;
    B cs2 = cs2a;
    bool bound = false;
    if constexpr (float_based<B>) {
        const B cs2b = K.cs2_rel * (v2 + ca2 + bt2);
        bound = cs2b > cs2a;
        cs2 = m::max_(cs2a, cs2b);
    }
    B fmc, cms, cf2, csl2;
    speeds<B>(cs2, ca2, bt2, fmc, cms, cf2, csl2);
    const B cf = m::sqrt_(cf2), csl = m::sqrt_(csl2), cs = m::sqrt_(cs2);
    const B dfs = fmc + cms;
    const bool brA = dfs >= K.eps_b2;
    B af = B(1), as = B(1), idf = B(0), qa = B(0), qs = B(0);
    if (brA) {
        idf = m::rcp_(dfs);
        qa = cms * idf;
        qs = fmc * idf;
        af = m::sqrt_(m::max_(qa, B(0)));
        as = m::sqrt_(m::max_(qs, B(0)));
    }
    const bool brB = btm > K.eps_b;
    B b1 = B(0.70710678118654752440), b2 = B(0.70710678118654752440), ib = B(0);
    if (brB) {
        ib = m::rsqrt_(btm);
        b1 = Bt1 * ib;
        b2 = Bt2 * ib;
    }
    const A sg = (Bn >= K.eps_b) ? A(1) : A(-1);
    const B sr = m::sqrt_(r);
    const B isr = sr * ir;
    const B bvB = b1 * vt1 + b2 * vt2;
    const B ics2B = m::rcp_(cs2);
    // the rest in the adjoint type
    const A Avn = (A)vn, Avt1 = (A)vt1, Avt2 = (A)vt2, ABt1 = (A)Bt1, ABt2 = (A)Bt2;
    const A Av2 = (A)v2, Acf = (A)cf, Acsl = (A)csl, Acs = (A)cs, Acf2 = (A)cf2, Acsl2 = (A)csl2, Acs2 = (A)cs2;
    const A Aaf = (A)af, Aas = (A)as, Ab1 = (A)b1, Ab2 = (A)b2, Asr = (A)sr, Aisr = (A)isr, Abv = (A)bvB;
    const A ics2 = (A)ics2B, pre = A(0.5) * ics2, gm1 = (A)K.gm1, g1 = (A)K.g1, g2 = (A)K.g2;
    const A tau = gm1 * ics2;
    const A Gf = Aaf * Acf * Avn - Aas * Acsl * sg * Abv;
    const A Gs = Aas * Acsl * Avn + Aaf * Acf * sg * Abv;
    const A k1 = -gm1 * Aaf, k2 = -gm1 * Aas;
    const A V[3] = {Avn, Avt1, Avt2};
    // ---- adjoints
    A lpre = 0, laf = 0, las = 0, lcf = 0, lcsl = 0, lcs = 0, lsr = 0, lisr = 0, lb1 = 0, lb2 = 0;
    A lGf = 0, lGs = 0, lGa = 0, lv2 = 0, lBt1 = 0, lBt2 = 0, lcf2 = 0, lcsl2 = 0, lcs2 = 0, ltau = 0;
    A lk1 = 0, lk2 = 0;
    A lv[3] = {0, 0, 0};
    // fast pair (modes 0, 1): L = Lc +- Ls, R = Rc +- Rs (rows 1, 2, 3, 6)
    {
        A lLc[7], lLs[4], lRc[7], lRs[4];
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            lLc[c] = lL[0][c] + lL[1][c];
            lRc[c] = lR[0][c] + lR[1][c];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) lLs[c] = lL[0][c] - lL[1][c];
        lRs[0] = lR[0][1] - lR[1][1];
        lRs[1] = lR[0][2] - lR[1][2];
        lRs[2] = lR[0][3] - lR[1][3];
        lRs[3] = lR[0][6] - lR[1][6];
        A l = lLc[0];
        lpre += l * g1 * Aaf * Av2;
        laf += l * pre * g1 * Av2;
        lv2 += l * pre * g1 * Aaf;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            l = lLc[1 + j];
            lpre += l * k1 * V[j];
            lk1 += l * pre * V[j];
            lv[j] += l * pre * k1;
        }
        {
            l = lLc[4];
            const A lt = l * pre;
            lpre += l * (k1 * ABt1 + Asr * Acs * Aas * Ab1);
            lk1 += lt * ABt1;
            lBt1 += lt * k1;
            lsr += lt * Acs * Aas * Ab1;
            lcs += lt * Asr * Aas * Ab1;
            las += lt * Asr * Acs * Ab1;
            lb1 += lt * Asr * Acs * Aas;
        }
        {
            l = lLc[5];
            const A lt = l * pre;
            lpre += l * (k1 * ABt2 + Asr * Acs * Aas * Ab2);
            lk1 += lt * ABt2;
            lBt2 += lt * k1;
            lsr += lt * Acs * Aas * Ab2;
            lcs += lt * Asr * Aas * Ab2;
            las += lt * Asr * Acs * Ab2;
            lb2 += lt * Asr * Acs * Aas;
        }
        l = lLc[6];
        lpre += l * gm1 * Aaf;
        laf += l * pre * gm1;
        l = lLs[0];
        lpre += l * Gf;
        lGf += l * pre;
        l = lLs[1];
        lpre -= l * Aaf * Acf;
        laf -= l * pre * Acf;
        lcf -= l * pre * Aaf;
        l = lLs[2];
        lpre += l * Acsl * Aas * Ab1 * sg;
        lcsl += l * pre * Aas * Ab1 * sg;
        las += l * pre * Acsl * Ab1 * sg;
        lb1 += l * pre * Acsl * Aas * sg;
        l = lLs[3];
        lpre += l * Acsl * Aas * Ab2 * sg;
        lcsl += l * pre * Aas * Ab2 * sg;
        las += l * pre * Acsl * Ab2 * sg;
        lb2 += l * pre * Acsl * Aas * sg;
        laf += lRc[0];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            l = lRc[1 + j];
            laf += l * V[j];
            lv[j] += l * Aaf;
        }
        l = lRc[4];
        lcs += l * Aas * Ab1 * Aisr;
        las += l * Acs * Ab1 * Aisr;
        lb1 += l * Acs * Aas * Aisr;
        lisr += l * Acs * Aas * Ab1;
        l = lRc[5];
        lcs += l * Aas * Ab2 * Aisr;
        las += l * Acs * Ab2 * Aisr;
        lb2 += l * Acs * Aas * Aisr;
        lisr += l * Acs * Aas * Ab2;
        l = lRc[6];
        laf += l * (A(0.5) * Av2 + Acf2 - g2 * Acs2);
        lv2 += l * Aaf * A(0.5);
        lcf2 += l * Aaf;
        lcs2 -= l * Aaf * g2;
        l = lRs[0];
        laf -= l * Acf;
        lcf -= l * Aaf;
        l = lRs[1];
        lcsl += l * Aas * Ab1 * sg;
        las += l * Acsl * Ab1 * sg;
        lb1 += l * Acsl * Aas * sg;
        l = lRs[2];
        lcsl += l * Aas * Ab2 * sg;
        las += l * Acsl * Ab2 * sg;
        lb2 += l * Acsl * Aas * sg;
        lGf -= lRs[3];
        laf -= gm1 * lk1;
    }
    // slow pair (modes 2, 3)
    {
        A lLc[7], lLs[4], lRc[7], lRs[4];
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            lLc[c] = lL[2][c] + lL[3][c];
            lRc[c] = lR[2][c] + lR[3][c];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) lLs[c] = lL[2][c] - lL[3][c];
        lRs[0] = lR[2][1] - lR[3][1];
        lRs[1] = lR[2][2] - lR[3][2];
        lRs[2] = lR[2][3] - lR[3][3];
        lRs[3] = lR[2][6] - lR[3][6];
        A l = lLc[0];
        lpre += l * g1 * Aas * Av2;
        las += l * pre * g1 * Av2;
        lv2 += l * pre * g1 * Aas;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            l = lLc[1 + j];
            lpre += l * k2 * V[j];
            lk2 += l * pre * V[j];
            lv[j] += l * pre * k2;
        }
        {
            l = lLc[4];
            const A lt = l * pre;
            lpre += l * (k2 * ABt1 - Asr * Acs * Aaf * Ab1);
            lk2 += lt * ABt1;
            lBt1 += lt * k2;
            lsr -= lt * Acs * Aaf * Ab1;
            lcs -= lt * Asr * Aaf * Ab1;
            laf -= lt * Asr * Acs * Ab1;
            lb1 -= lt * Asr * Acs * Aaf;
        }
        {
            l = lLc[5];
            const A lt = l * pre;
            lpre += l * (k2 * ABt2 - Asr * Acs * Aaf * Ab2);
            lk2 += lt * ABt2;
            lBt2 += lt * k2;
            lsr -= lt * Acs * Aaf * Ab2;
            lcs -= lt * Asr * Aaf * Ab2;
            laf -= lt * Asr * Acs * Ab2;
            lb2 -= lt * Asr * Acs * Aaf;
        }
        l = lLc[6];
        lpre += l * gm1 * Aas;
        las += l * pre * gm1;
        l = lLs[0];
        lpre += l * Gs;
        lGs += l * pre;
        l = lLs[1];
        lpre -= l * Aas * Acsl;
        las -= l * pre * Acsl;
        lcsl -= l * pre * Aas;
        l = lLs[2];
        lpre -= l * Acf * Aaf * Ab1 * sg;
        lcf -= l * pre * Aaf * Ab1 * sg;
        laf -= l * pre * Acf * Ab1 * sg;
        lb1 -= l * pre * Acf * Aaf * sg;
        l = lLs[3];
        lpre -= l * Acf * Aaf * Ab2 * sg;
        lcf -= l * pre * Aaf * Ab2 * sg;
        laf -= l * pre * Acf * Ab2 * sg;
        lb2 -= l * pre * Acf * Aaf * sg;
        las += lRc[0];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            l = lRc[1 + j];
            las += l * V[j];
            lv[j] += l * Aas;
        }
        l = lRc[4];
        lcs -= l * Aaf * Ab1 * Aisr;
        laf -= l * Acs * Ab1 * Aisr;
        lb1 -= l * Acs * Aaf * Aisr;
        lisr -= l * Acs * Aaf * Ab1;
        l = lRc[5];
        lcs -= l * Aaf * Ab2 * Aisr;
        laf -= l * Acs * Ab2 * Aisr;
        lb2 -= l * Acs * Aaf * Aisr;
        lisr -= l * Acs * Aaf * Ab2;
        l = lRc[6];
        las += l * (A(0.5) * Av2 + Acsl2 - g2 * Acs2);
        lv2 += l * Aas * A(0.5);
        lcsl2 += l * Aas;
        lcs2 -= l * Aas * g2;
        l = lRs[0];
        las -= l * Acsl;
        lcsl -= l * Aas;
        l = lRs[1];
        lcf -= l * Aaf * Ab1 * sg;
        laf -= l * Acf * Ab1 * sg;
        lb1 -= l * Acf * Aaf * sg;
        l = lRs[2];
        lcf -= l * Aaf * Ab2 * sg;
        laf -= l * Acf * Ab2 * sg;
        lb2 -= l * Acf * Aaf * sg;
        lGs -= lRs[3];
        las -= gm1 * lk2;
    }
    // Alfven pair (modes 4, 5)
    {
        const A ll0 = lL[4][0] + lL[5][0], ll2 = lL[4][2] + lL[5][2], ll3 = lL[4][3] + lL[5][3];
        const A ll4 = lL[4][4] - lL[5][4], ll5 = lL[4][5] - lL[5][5];
        lGa += A(0.5) * ll0;
        lb2 -= A(0.5) * sg * ll2;
        lb1 += A(0.5) * sg * ll3;
        lsr -= A(0.5) * Ab2 * ll4;
        lb2 -= A(0.5) * Asr * ll4;
        lsr += A(0.5) * Ab1 * ll5;
        lb1 += A(0.5) * Asr * ll5;
        const A r2 = lR[4][2] + lR[5][2], r3 = lR[4][3] + lR[5][3], r4 = lR[4][4] - lR[5][4];
        const A r5 = lR[4][5] - lR[5][5], r6 = lR[4][6] + lR[5][6];
        lb2 -= sg * r2;
        lb1 += sg * r3;
        lb2 -= Aisr * r4;
        lisr -= Ab2 * r4;
        lb1 += Aisr * r5;
        lisr += Ab1 * r5;
        lGa -= r6;
    }
    // entropy (mode 6)
    {
        A l = lL[6][0];
        ltau -= A(0.5) * Av2 * l;
        lv2 -= A(0.5) * tau * l;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            l = lL[6][1 + j];
            ltau += l * V[j];
            lv[j] += l * tau;
        }
        ltau += lL[6][4] * ABt1;
        lBt1 += lL[6][4] * tau;
        ltau += lL[6][5] * ABt2;
        lBt2 += lL[6][5] * tau;
        ltau -= lL[6][6];
#pragma unroll
        for (int j = 0; j < 3; ++j) lv[j] += lR[6][1 + j];
        lv2 += A(0.5) * lR[6][6];
    }
    // ---- the scalars, backwards
    const A lics2 = gm1 * ltau + A(0.5) * lpre;
    lcs2 -= ics2 * (ics2 * lics2);
    las += lGs * Acsl * Avn;
    lcsl += lGs * Aas * Avn;
    lv[0] += lGs * Aas * Acsl;
    laf += lGs * Acf * sg * Abv;
    lcf += lGs * Aaf * sg * Abv;
    A lbv = lGs * Aaf * Acf * sg;
    // Ga = sg (b2 vt1 - b1 vt2)
    lb2 += lGa * sg * Avt1;
    lv[1] += lGa * sg * Ab2;
    lb1 -= lGa * sg * Avt2;
    lv[2] -= lGa * sg * Ab1;
    laf += lGf * Acf * Avn;
    lcf += lGf * Aaf * Avn;
    lv[0] += lGf * Aaf * Acf;
    las -= lGf * Acsl * sg * Abv;
    lcsl -= lGf * Aas * sg * Abv;
    lbv -= lGf * Aas * Acsl * sg;
    lb1 += lbv * Avt1;
    lv[1] += lbv * Ab1;
    lb2 += lbv * Avt2;
    lv[2] += lbv * Ab2;
    const A Air = (A)ir;
    A lir = lisr * Asr;
    lsr += lisr * Air;
    A lr = sr > B(0) ? lsr * A(0.5) / Asr : A(0);
    A lbtm = A(0);
    if (brB) {
        const A Aib = (A)ib;
        lBt1 += lb1 * Aib;
        lBt2 += lb2 * Aib;
        const A lib = lb1 * ABt1 + lb2 * ABt2;
        lbtm -= A(0.5) * Aib * (Aib * (Aib * lib));
    }
    A lfmc = A(0), lcms = A(0);
    if (brA) {
        const A lqa = qa > B(0) ? laf * A(0.5) / Aaf : A(0);
        const A lqs = qs > B(0) ? las * A(0.5) / Aas : A(0);
        const A Aidf = (A)idf;
        lcms += lqa * Aidf;
        lfmc += lqs * Aidf;
        const A lidf = lqa * (A)cms + lqs * (A)fmc;
        const A ldfs = -Aidf * (Aidf * lidf);
        lfmc += ldfs;
        lcms += ldfs;
    }
    if (cs > B(0)) lcs2 += lcs * A(0.5) / Acs;
    if (csl > B(0)) lcsl2 += lcsl * A(0.5) / Acsl;
    if (cf > B(0)) lcf2 += lcf * A(0.5) / Acf;
    A lca2 = A(0), lbt2 = A(0);
    speeds_rev<B, A>(cs2, ca2, bt2, lfmc, lcms, lcf2, lcsl2, lcs2, lca2, lbt2);
    A lP = A(0);
    if (bound) {
        const A t = (A)K.cs2_rel * lcs2;
        lv2 += t;
        lca2 += t;
        lbt2 += t;
    } else {
        lP += (A)K.gamma * Air * lcs2;
        lir += (A)K.gamma * (A)P * lcs2;
    }
    lv[0] += A(2) * Avn * lv2;
    lv[1] += A(2) * Avt1 * lv2;
    lv[2] += A(2) * Avt2 * lv2;
    lbtm += Air * lbt2;
    lir += (A)btm * lbt2;
    lBt1 += A(2) * ABt1 * lbtm;
    lBt2 += A(2) * ABt2 * lbtm;
    const A lBn = A(2) * (A)Bn * Air * lca2;
    lir += (A)Bn * (A)Bn * lca2;
    lr -= Air * (Air * lir);
    lw[0] = lr;
    lw[1] = lv[0];
    lw[2] = lv[1];
    lw[3] = lv[2];
    lw[4] = lBn;
    lw[5] = lBt1;
    lw[6] = lBt2;
    lw[7] = lP;
}

// phi_N(a, b, c, d) of Sec. 2.2 (the weights of the forward step: JS, or
// WENO-Z with the ratio clamped at 1e18 in float) and its gradient in (a, b,
// c, d), by hand: smoothness indicators -> weights (through tau for WENO-Z)
// -> the two interpolants, run backwards.
template <typename B, int VAR>
__device__ __forceinline__ void phi_n_grad(B a, B b, B c, B d, B eps, B &phi, B (&g)[4]) {
    const B x0 = a - b, x1 = a - B(3) * b, y0 = b - c, y1 = b + c, z0 = c - d, z1 = B(3) * c - d;
    const B IS0 = B(13) * x0 * x0 + B(3) * x1 * x1;
    const B IS1 = B(13) * y0 * y0 + B(3) * y1 * y1;
    const B IS2 = B(13) * z0 * z0 + B(3) * z1 * z1;
    const B s[3] = {eps + IS0, eps + IS1, eps + IS2};
    const B dk[3] = {B(1), B(6), B(3)};
    B al[3], r[3], t = B(0);
    bool clamped[3] = {false, false, false};
    if constexpr (VAR == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) al[k] = dk[k] / (s[k] * s[k]);
    } else {
        t = IS0 - IS2;
        const B tau = t >= B(0) ? t : -t;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            r[k] = tau / s[k];
            if constexpr (float_based<B>) {
                if (r[k] > B(1.0e18)) {
                    r[k] = B(1.0e18);
                    clamped[k] = true;
                }
            }
            al[k] = dk[k] * (B(1) + r[k] * r[k]);
        }
    }
    const B S = al[0] + al[1] + al[2];
    const B w0 = al[0] / S, w2 = al[2] / S;
    const B t1 = a - B(2) * b + c, t2 = b - B(2) * c + d;
    phi = w0 * B(1.0 / 3.0) * t1 + (w2 - B(0.5)) * B(1.0 / 6.0) * t2;
    // backwards, with d(phi) = 1
    const B lw0 = t1 * B(1.0 / 3.0), lw2 = t2 * B(1.0 / 6.0);
    const B lt1 = w0 * B(1.0 / 3.0), lt2 = (w2 - B(0.5)) * B(1.0 / 6.0);
    const B common = (lw0 * w0 + lw2 * w2) / S;
    const B la[3] = {lw0 / S - common, -common, lw2 / S - common};
    B lIS[3];
    if constexpr (VAR == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) lIS[k] = la[k] * (B(-2) * al[k] / s[k]);
    } else {
        B ltau = B(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const B lr = clamped[k] ? B(0) : la[k] * dk[k] * B(2) * r[k];
            ltau = ltau + lr / s[k];
            lIS[k] = -lr * r[k] / s[k];
        }
        const B lt = t >= B(0) ? ltau : -ltau;
        lIS[0] = lIS[0] + lt;
        lIS[2] = lIS[2] - lt;
    }
    g[0] = lIS[0] * (B(26) * x0 + B(6) * x1) + lt1;
    g[1] = lIS[0] * (B(-26) * x0 - B(18) * x1) + lIS[1] * (B(26) * y0 + B(6) * y1) - B(2) * lt1 + lt2;
    g[2] = lIS[1] * (B(-26) * y0 + B(6) * y1) + lIS[2] * (B(26) * z0 + B(18) * z1) + lt1 - B(2) * lt2;
    g[3] = lIS[2] * (B(-26) * z0 - B(6) * z1) + lt2;
}

// weno_field (Eq. FWENO for one characteristic field) and its gradient in
// its eleven projections and in alpha.
template <typename B, int VAR>
__device__ __forceinline__ void weno_field_grad(const B (&P)[11], B alpha, B eps4, B &phi, B (&gP)[11], B &galpha) {
    B p[5], q[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        p[j] = P[1 + j] + alpha * P[6 + j];
        q[j] = P[1 + j] - alpha * P[6 + j];
    }
    B fp, fq, gpa[4], gqa[4];
    phi_n_grad<B, VAR>(p[0], p[1], p[2], p[3], eps4, fp, gpa);
    phi_n_grad<B, VAR>(q[4], q[3], q[2], q[1], eps4, fq, gqa);
    phi = P[0] + B(0.5) * (fq - fp);
    B gp[5], gq[5];
#pragma unroll
    for (int j = 0; j < 4; ++j) gp[j] = B(-0.5) * gpa[j];
    gp[4] = B(0);
    gq[0] = B(0);
#pragma unroll
    for (int j = 1; j < 5; ++j) gq[j] = B(0.5) * gqa[4 - j];
    gP[0] = B(1);
    galpha = B(0);
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        gP[1 + j] = gp[j] + gq[j];
        gP[6 + j] = alpha * (gp[j] - gq[j]);
        galpha = galpha + P[6 + j] * (gp[j] - gq[j]);
    }
}

// Reverse of cell_fill<B, AX>: given the adjoints lq of a cell's 23
// quantities, the adjoints of its eight inputs (rho, m_x, m_y, m_z, E, B_x,
// B_y, B_z) in out.  The primitives and the flux are differentiated by hand
// (Eq. P and Eq. fluxes), and so are the three wave speeds when their
// adjoints are not zero (the two cells next to the face), through
// speeds_rev.  The floors, when they apply, cut the dependence as in the
// forward step.
template <typename B, typename A, int AX>
__device__ __forceinline__ void cell_fill_adjoint(const B (&in)[8], const A (&lq)[NCQ], const Phys<B> &K,
                                                  A (&out)[8]) {
    constexpr int n = AX, t1 = (AX + 1) % 3, t2 = (AX + 2) % 3;
    const B rho = in[0], mn = in[1 + n], m1 = in[1 + t1], m2 = in[1 + t2], E = in[4];
    const B Bn = in[5 + n], B1 = in[5 + t1], B2 = in[5 + t2];
    B r = rho;
    bool rfloor = false, pfloor = false;
    if (K.floors && r < K.rho_min) {
        r = K.rho_min;
        rfloor = true;
    }
    const B ir = M<B>::rcp_(r);
    const A vn = (A)(mn * ir), v1 = (A)(m1 * ir), v2 = (A)(m2 * ir);
    const A vv = vn * vn + v1 * v1 + v2 * v2;
    const A BB = (A)Bn * (A)Bn + (A)B1 * (A)B1 + (A)B2 * (A)B2;
    B P = K.gm1 * (E - B(0.5) * r * (B)vv - B(0.5) * (B)BB);
    if (K.floors && P < K.p_min) {
        P = K.p_min;
        pfloor = true;
    }
    const A rA = (A)r, PA = (A)P, EA = (A)E, bn = (A)Bn, b1 = (A)B1, b2 = (A)B2;
    const A Pt = PA + A(0.5) * BB;
    const A vB = vn * bn + v1 * b1 + v2 * b2;
    A lr = lq[C_RHO], lvn = lq[C_VN], lv1 = lq[C_VT1], lv2 = lq[C_VT2];
    A lBn = lq[C_BN], lB1 = lq[C_BT1], lB2 = lq[C_BT2], lP = lq[C_P];
    A lE = lq[C_E], lmn = lq[C_MN], lm1 = lq[C_MT1], lm2 = lq[C_MT2], lrho = lq[C_RHOQ];
    A lPt = A(0), lvB = A(0);
    {   // F0 = r vn, F1 = r vn^2 + Pt - Bn^2, F2 = r vn v1 - Bn B1, F3 = r vn v2 - Bn B2
        const A f0 = lq[C_F0], f1 = lq[C_F1], f2 = lq[C_F2], f3 = lq[C_F3];
        lr += f0 * vn + f1 * vn * vn + f2 * vn * v1 + f3 * vn * v2;
        lvn += f0 * rA + f1 * A(2) * rA * vn + f2 * rA * v1 + f3 * rA * v2;
        lPt += f1;
        lBn -= f1 * A(2) * bn + f2 * b1 + f3 * b2;
        lv1 += f2 * rA * vn;
        lv2 += f3 * rA * vn;
        lB1 -= f2 * bn;
        lB2 -= f3 * bn;
    }
    {   // F4 = B1 vn - Bn v1, F5 = B2 vn - Bn v2, F6 = (E + Pt) vn - Bn vB
        const A f4 = lq[C_F4], f5 = lq[C_F5], f6 = lq[C_F6];
        lB1 += f4 * vn;
        lB2 += f5 * vn;
        lvn += f4 * b1 + f5 * b2 + f6 * (EA + Pt);
        lBn -= f4 * v1 + f5 * v2 + f6 * vB;
        lv1 -= f4 * bn;
        lv2 -= f5 * bn;
        lE += f6 * vn;
        lPt += f6 * vn;
        lvB -= f6 * bn;
    }
    // vB = vn Bn + v1 B1 + v2 B2; Pt = P + BB/2
    lvn += lvB * bn;
    lv1 += lvB * b1;
    lv2 += lvB * b2;
    lBn += lvB * vn + lPt * bn;
    lB1 += lvB * v1 + lPt * b1;
    lB2 += lvB * v2 + lPt * b2;
    lP += lPt;
    // wave speeds c_f, c_A, c_slow of the cell from (r, P, Bn, B1, B2),
    // reversed by hand (Eqs. slow/fast through speeds_rev; |Bn| and sqrt(0)
    // take the sign of Bn and the subgradient 0)
    const A lcf = lq[C_CF], lca = lq[C_CA], lcs = lq[C_CSL];
    if (lcf != A(0) || lca != A(0) || lcs != A(0)) {
        using mb = M<B>;
        const B irr = mb::rcp_(r);
        const B cs2 = K.gamma * P * irr, ca2 = Bn * Bn * irr, bt2 = (B1 * B1 + B2 * B2) * irr;
        B fmc, cms, cf2, csl2;
        speeds<B>(cs2, ca2, bt2, fmc, cms, cf2, csl2);
        const B cf = mb::sqrt_(cf2), csl = mb::sqrt_(csl2), sr = mb::sqrt_(r);
        const A lcf2 = cf > B(0) ? lcf * A(0.5) / (A)cf : A(0);
        const A lcsl2 = csl > B(0) ? lcs * A(0.5) / (A)csl : A(0);
        A lcs2 = A(0), lca2 = A(0), lbt2 = A(0);
        speeds_rev<B, A>(cs2, ca2, bt2, A(0), A(0), lcf2, lcsl2, lcs2, lca2, lbt2);
        // c_A = |Bn| (sqrt(r) / r)
        const A Airr = (A)irr, Asr = (A)sr;
        const A sgn = Bn >= B(0) ? A(1) : A(-1);
        lBn += lca * sgn * Asr * Airr;
        const A lq_ = lca * sgn * (A)Bn;              // adjoint of sqrt(r) / r
        A lirr = lq_ * Asr;
        const A lsr = lq_ * Airr;
        if (sr > B(0)) lr += lsr * A(0.5) / Asr;
        // cs2 = gamma P / r, ca2 = Bn^2 / r, bt2 = (B1^2 + B2^2) / r
        lP += (A)K.gamma * Airr * lcs2;
        lirr += (A)K.gamma * (A)P * lcs2;
        lBn += A(2) * (A)Bn * Airr * lca2;
        lirr += (A)Bn * (A)Bn * lca2;
        lB1 += A(2) * (A)B1 * Airr * lbt2;
        lB2 += A(2) * (A)B2 * Airr * lbt2;
        lirr += ((A)B1 * (A)B1 + (A)B2 * (A)B2) * lbt2;
        lr -= Airr * (Airr * lirr);
    }
    // P = gm1 (E - r vv / 2 - BB / 2)
    if (!pfloor) {
        const A gl = (A)K.gm1 * lP;
        lE += gl;
        lr -= A(0.5) * vv * gl;
        lvn -= rA * vn * gl;
        lv1 -= rA * v1 * gl;
        lv2 -= rA * v2 * gl;
        lBn -= bn * gl;
        lB1 -= b1 * gl;
        lB2 -= b2 * gl;
    }
    // v = m / r
    const A irA = (A)ir;
    lmn += lvn * irA;
    lm1 += lv1 * irA;
    lm2 += lv2 * irA;
    lr -= (lvn * vn + lv1 * v1 + lv2 * v2) * irA;
    if (!rfloor) lrho += lr;
    out[0] = lrho;
    out[1 + n] = lmn;
    out[1 + t1] = lm1;
    out[1 + t2] = lm2;
    out[4] = lE;
    out[5 + n] = lBn;
    out[5 + t1] = lB1;
    out[5 + t2] = lB2;
}

// Reverse mode of the face function.  Face p (the interface between cell p
// and its successor along AX) reads stencil cells p-2 .. p+3 (inputs rho,
// m_x, m_y, m_z, E, B_x, B_y, B_z each); its outputs are the five lab-order
// face fluxes and the two transport fluxes.  One primal evaluation (the
// formulas of cell_fill and face_flux), then the transposes of the linear
// parts (stencil combinations, projection on the left eigenvectors,
// back-projection on the right ones), of phi_N (phi_n_grad) and of the cell
// recovery (cell_fill_adjoint) and of the eigenvectors (eigen7_rev), all
// written by hand.  Branches follow the primal values (the derivative of the
// branch the forward step takes).  The 48 contributions
// d(lam . outputs)/d(input) go to cb; adjoints accumulate in double (float
// in the float path, whose Jacobians are float).
template <int AX, typename B, int VAR>
__global__ void __launch_bounds__(128) adj_face_kernel(AdjSweepArgs<B> a) {
    using A = typename std::conditional<std::is_same<B, float>::value, float, double>::type;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long n = (long long)nx * ny * nz;
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int i = (int)(p % nx);
    const long long r = p / nx;
    const int j = (int)(r % ny), k = (int)(r / ny);
    B in[6][8];
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        const int ii = AX == 0 ? wrapi(i - 2 + s, nx) : i;
        const int jj = AX == 1 ? wrapi(j - 2 + s, ny) : j;
        const int kk = AX == 2 ? wrapi(k - 2 + s, nz) : k;
        const size_t g = (size_t)ii + (size_t)nx * ((size_t)jj + (size_t)ny * (size_t)kk);
#pragma unroll
        for (int f = 0; f < 5; ++f) in[s][f] = a.q[f][g];
#pragma unroll
        for (int f = 0; f < 3; ++f) in[s][5 + f] = a.bc[f][g];
    }
    const A lam5 = from_double<A>(a.lamS[0][p]), lam6 = from_double<A>(a.lamS[1][p]);
    // adjoint of the frame flux Ff (s1 = Ff[4] + bvt1, s2 = Ff[5] + bvt2)
    A lFf[7];
    lFf[0] = from_double<A>(a.lamF[0][p]);
    lFf[1] = from_double<A>(a.lamF[1 + AX][p]);
    lFf[2] = from_double<A>(a.lamF[1 + (AX + 1) % 3][p]);
    lFf[3] = from_double<A>(a.lamF[1 + (AX + 2) % 3][p]);
    lFf[4] = (A)lam5;
    lFf[5] = (A)lam6;
    lFf[6] = from_double<A>(a.lamF[4][p]);
    const Phys<B> K = a.K;
    bool bad = false, hit = false;
    B cq[NCQ * 6];
#pragma unroll 1
    for (int c = 0; c < 6; ++c)
        cell_fill<B, AX>(cq + c, 6, in[c][0], in[c][1], in[c][2], in[c][3], in[c][4], in[c][5], in[c][6], in[c][7], K,
                         bad, hit);
#define Q(q, kk) cq[(q) * 6 + (kk)]
    constexpr int qU[7] = {C_RHOQ, C_MN, C_MT1, C_MT2, C_BT1, C_BT2, C_E};
    B X[11][7];
#pragma unroll
    for (int c = 0; c < 7; ++c) {
        const B f0 = Q(C_F0 + c, 0), f1 = Q(C_F0 + c, 1), f2 = Q(C_F0 + c, 2), f3 = Q(C_F0 + c, 3), f4 = Q(C_F0 + c, 4),
                f5 = Q(C_F0 + c, 5);
        X[0][c] = (B(7) * (f2 + f3) - (f1 + f4)) * B(1.0 / 12.0);
        X[1][c] = f1 - f0;
        X[2][c] = f2 - f1;
        X[3][c] = f3 - f2;
        X[4][c] = f4 - f3;
        X[5][c] = f5 - f4;
        const B u0 = Q(qU[c], 0), u1 = Q(qU[c], 1), u2 = Q(qU[c], 2), u3 = Q(qU[c], 3), u4 = Q(qU[c], 4),
                u5 = Q(qU[c], 5);
        X[6][c] = u1 - u0;
        X[7][c] = u2 - u1;
        X[8][c] = u3 - u2;
        X[9][c] = u4 - u3;
        X[10][c] = u5 - u4;
    }
    // LF speeds alpha(m) = max over cells 2, 3 of |v_n + sgn c|, with the
    // cell and sign that attain it (the branch the forward step takes)
    constexpr int cq_of_mode[7] = {C_CF, C_CF, C_CSL, C_CSL, C_CA, C_CA, -1};
    constexpr int sgn_of_mode[7] = {-1, 1, -1, 1, -1, 1, 0};
    B alpha[7];
    int acell[7];
    B asign[7];
#pragma unroll
    for (int mo = 0; mo < 7; ++mo) {
        const B c2 = cq_of_mode[mo] >= 0 ? Q(cq_of_mode[mo], 2) : B(0);
        const B c3 = cq_of_mode[mo] >= 0 ? Q(cq_of_mode[mo], 3) : B(0);
        const B x2 = Q(C_VN, 2) + B(sgn_of_mode[mo]) * c2, x3 = Q(C_VN, 3) + B(sgn_of_mode[mo]) * c3;
        const B a2 = x2 >= B(0) ? x2 : -x2, a3 = x3 >= B(0) ? x3 : -x3;
        acell[mo] = a2 >= a3 ? 2 : 3;
        alpha[mo] = a2 >= a3 ? a2 : a3;
        asign[mo] = (a2 >= a3 ? x2 : x3) >= B(0) ? B(1) : B(-1);
    }
    // eigenvectors at the interface state (values); their dependence on the
    // state is reversed by eigen7_rev after the mode loop
    B wv[8];
    const int prim[8] = {C_RHO, C_VN, C_VT1, C_VT2, C_BN, C_BT1, C_BT2, C_P};
#pragma unroll
    for (int t = 0; t < 8; ++t) wv[t] = B(0.5) * (Q(prim[t], 2) + Q(prim[t], 3));
    B Lv[7][7], Rv[7][7];
    eigen7<B>(wv, K, Lv, Rv);
    A lLm[7][7], lRm[7][7];
    const B eps4 = B(4) * K.eps_w;
    A lX[11][7];
#pragma unroll
    for (int x = 0; x < 11; ++x)
#pragma unroll
        for (int c = 0; c < 7; ++c) lX[x][c] = A(0);
    A lw[8];
    A lalpha[7];
#pragma unroll 1
    for (int mo = 0; mo < 7; ++mo) {
        B Pm[11];
#pragma unroll
        for (int x = 0; x < 11; ++x) {
            B acc = Lv[mo][0] * X[x][0];
#pragma unroll
            for (int c = 1; c < 7; ++c) acc = acc + Lv[mo][c] * X[x][c];
            Pm[x] = acc;
        }
        B phi, gP[11], ga;
        weno_field_grad<B, VAR>(Pm, alpha[mo], eps4, phi, gP, ga);
        A lphi = A(0);
#pragma unroll
        for (int c = 0; c < 7; ++c) lphi += (A)Rv[mo][c] * lFf[c];
        lalpha[mo] = lphi * (A)ga;
        A lL[7] = {0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int x = 0; x < 11; ++x) {
            const A lp = lphi * (A)gP[x];
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                lX[x][c] += lp * (A)Lv[mo][c];
                lL[c] += lp * (A)X[x][c];
            }
        }
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            lLm[mo][c] = lL[c];
            lRm[mo][c] = (A)phi * lFf[c];
        }
    }
    eigen7_rev<B, A>(wv, K, lLm, lRm, lw);
    // adjoints of the cells' quantities
    A lq[6][NCQ];
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int q = 0; q < NCQ; ++q) lq[c][q] = A(0);
#pragma unroll
    for (int c = 0; c < 7; ++c) {
        // X[0] = (7 (f2 + f3) - (f1 + f4)) / 12, X[1 + k] = f_{k+1} - f_k, X[6 + k] = u_{k+1} - u_k
        const A l0 = lX[0][c] * A(1.0 / 12.0);
        lq[1][C_F0 + c] -= l0;
        lq[2][C_F0 + c] += A(7) * l0;
        lq[3][C_F0 + c] += A(7) * l0;
        lq[4][C_F0 + c] -= l0;
#pragma unroll
        for (int kk = 0; kk < 5; ++kk) {
            lq[kk + 1][C_F0 + c] += lX[1 + kk][c];
            lq[kk][C_F0 + c] -= lX[1 + kk][c];
            lq[kk + 1][qU[c]] += lX[6 + kk][c];
            lq[kk][qU[c]] -= lX[6 + kk][c];
        }
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        lq[2][prim[t]] += A(0.5) * lw[t];
        lq[3][prim[t]] += A(0.5) * lw[t];
    }
#pragma unroll
    for (int mo = 0; mo < 7; ++mo) {
        const A g = lalpha[mo] * (A)asign[mo];
        lq[acell[mo]][C_VN] += g;
        if (cq_of_mode[mo] >= 0) lq[acell[mo]][cq_of_mode[mo]] += g * A(sgn_of_mode[mo]);
    }
    // transport fluxes bvt = (B_n v_t (cell 2) + B_n v_t (cell 3)) / 2
#pragma unroll
    for (int c = 2; c <= 3; ++c) {
        lq[c][C_BN] += A(0.5) * (lam5 * (A)Q(C_VT1, c) + lam6 * (A)Q(C_VT2, c));
        lq[c][C_VT1] += A(0.5) * lam5 * (A)Q(C_BN, c);
        lq[c][C_VT2] += A(0.5) * lam6 * (A)Q(C_BN, c);
    }
#undef Q
    // each cell's quantities back to its eight inputs
#pragma unroll 1
    for (int c = 0; c < 6; ++c) {
        A g[8];
        cell_fill_adjoint<B, A, AX>(in[c], lq[c], K, g);
#pragma unroll
        for (int v = 0; v < 8; ++v) a.cb[(size_t)(c * 8 + v) * (size_t)n + (size_t)p] = to_double(g[v]);
    }
}

// Cell p collects, in a fixed order, the contributions of the six faces whose
// stencils hold it (face p - s + 2 holds it as stencil cell s):
// lamq[v] += ... (v < 5), lambc[v - 5] += ... (v >= 5).
template <int AX>
__global__ void __launch_bounds__(256) adj_gather_kernel(int nx, int ny, int nz, const double *__restrict__ cb,
                                                         double *lq0, double *lq1, double *lq2, double *lq3,
                                                         double *lq4, double *lb0, double *lb1, double *lb2) {
    const long long n = (long long)nx * ny * nz;
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int i = (int)(p % nx);
    const long long r = p / nx;
    const int j = (int)(r % ny), k = (int)(r / ny);
    size_t face[6];
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        const int ii = AX == 0 ? wrapi(i + 2 - s, nx) : i;
        const int jj = AX == 1 ? wrapi(j + 2 - s, ny) : j;
        const int kk = AX == 2 ? wrapi(k + 2 - s, nz) : k;
        face[s] = (size_t)ii + (size_t)nx * ((size_t)jj + (size_t)ny * (size_t)kk);
    }
    double *out[8] = {lq0, lq1, lq2, lq3, lq4, lb0, lb1, lb2};
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        double acc = 0.0;
#pragma unroll
        for (int s = 0; s < 6; ++s) acc += cb[(size_t)(s * 8 + v) * (size_t)n + face[s]];
        out[v][p] += acc;
    }
}

// ---------------------------------------------------------------- linear parts

struct AdjGrid {
    int nx, ny, nz;
    double rdx, rdy, rdz;
    __device__ __forceinline__ size_t at(int i, int j, int k) const {
        return (size_t)wrapi(i, nx) + (size_t)nx * ((size_t)wrapi(j, ny) + (size_t)ny * (size_t)wrapi(k, nz));
    }
};

__device__ __forceinline__ bool adj_cell(const AdjGrid &g, int &i, int &j, int &k, size_t &p) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= n) return false;
    i = (int)(q % g.nx);
    const long long r = q / g.nx;
    j = (int)(r % g.ny);
    k = (int)(r / g.ny);
    p = (size_t)q;
    return true;
}

// stage sources: lamD = cf lamq_fin + cn lamq_next, mu = cf lamb_fin + cn lamb_next
// (mu is the adjoint of the stage's face-field increment dt-scaled curl Omega)
static __global__ void __launch_bounds__(256) adj_sources_kernel(long long n, double cf, double cn,
                                                                 const double *__restrict__ lq_fin,
                                                                 const double *__restrict__ lb_fin,
                                                                 const double *__restrict__ lq_next,
                                                                 const double *__restrict__ lb_next, double *lamD,
                                                                 double *mu) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= n) return;
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        const size_t o = (size_t)f * (size_t)n + (size_t)p;
        lamD[o] = cf * lq_fin[o] + (lq_next ? cn * lq_next[o] : 0.0);
    }
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        const size_t o = (size_t)f * (size_t)n + (size_t)p;
        mu[o] = cf * lb_fin[o] + (lb_next ? cn * lb_next[o] : 0.0);
    }
}

// lamO = curl^T mu for the face update of Sec. 2.3:
//   db_x = -(O_x - O_x(j-1)) rdy + (O_z - O_z(k-1)) rdz
//   db_y = -(O_y - O_y(k-1)) rdz + (O_x - O_x(i-1)) rdx
//   db_z = -(O_z - O_z(i-1)) rdx + (O_y - O_y(j-1)) rdy
static __global__ void __launch_bounds__(256) adj_curl_kernel(AdjGrid g, const double *__restrict__ mu, double *lamO) {
    int i, j, k;
    size_t p;
    if (!adj_cell(g, i, j, k, p)) return;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const double *mx = mu, *my = mu + n, *mz = mu + 2 * n;
    lamO[p] = g.rdy * (mx[g.at(i, j + 1, k)] - mx[p]) + g.rdx * (my[p] - my[g.at(i + 1, j, k)]);
    lamO[n + p] = g.rdz * (my[g.at(i, j, k + 1)] - my[p]) + g.rdy * (mz[p] - mz[g.at(i, j + 1, k)]);
    lamO[2 * n + p] = g.rdz * (mx[p] - mx[g.at(i, j, k + 1)]) + g.rdx * (mz[g.at(i + 1, j, k)] - mz[p]);
}

// Flux adjoints from lamD (transpose of Eq. num) and lamO (transpose of the
// EMF averages of Eqs. ox1-ox3):
//   O_x = (g*_x + g*_x(i+1))/2 - (f*_y + f*_y(j+1))/2
//   O_y = (h*_y + h*_y(j+1))/2 - (g*_z + g*_z(k+1))/2
//   O_z = (f*_z + f*_z(k+1))/2 - (h*_x + h*_x(i+1))/2
// lamF: 15 planes (axis-major: x fields 0..4, y, z); lamS: 6 planes
// (f*_y, f*_z, g*_z, g*_x, h*_x, h*_y, the storage order of the sweeps).
static __global__ void __launch_bounds__(256) adj_flux_kernel(AdjGrid g, const double *__restrict__ lamD,
                                                              const double *__restrict__ lamO, double *lamF,
                                                              double *lamS) {
    int i, j, k;
    size_t p;
    if (!adj_cell(g, i, j, k, p)) return;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const size_t px = g.at(i + 1, j, k), py = g.at(i, j + 1, k), pz = g.at(i, j, k + 1);
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        const double *L = lamD + (size_t)f * n;
        const double c = L[p];
        lamF[(size_t)f * n + p] = g.rdx * (L[px] - c);
        lamF[(size_t)(5 + f) * n + p] = g.rdy * (L[py] - c);
        lamF[(size_t)(10 + f) * n + p] = g.rdz * (L[pz] - c);
    }
    const double *Ox = lamO, *Oy = lamO + n, *Oz = lamO + 2 * n;
    const double ox = Ox[p], oy = Oy[p], oz = Oz[p];
    lamS[p] = -0.5 * (ox + Ox[g.at(i, j - 1, k)]);              // f*_y
    lamS[n + p] = 0.5 * (oz + Oz[g.at(i, j, k - 1)]);           // f*_z
    lamS[2 * n + p] = -0.5 * (oy + Oy[g.at(i, j, k - 1)]);      // g*_z
    lamS[3 * n + p] = 0.5 * (ox + Ox[g.at(i - 1, j, k)]);       // g*_x
    lamS[4 * n + p] = -0.5 * (oz + Oz[g.at(i - 1, j, k)]);      // h*_x
    lamS[5 * n + p] = 0.5 * (oy + Oy[g.at(i, j - 1, k)]);       // h*_y
}

// Transpose of the fourth-order face -> centre interpolation of Sec. 2.3,
// B_d(i) = (9 (b_d(i-1) + b_d(i)) - (b_d(i-2) + b_d(i+1))) / 16 along d:
// lamb_d(m) = (9 (lamB(m+1) + lamB(m)) - (lamB(m+2) + lamB(m-1))) / 16.
// Writes lamb (3 planes) and adds lamq, lamb into the step's outputs.
static __global__ void __launch_bounds__(256) adj_interp_kernel(AdjGrid g, const double *__restrict__ lamBc,
                                                                const double *__restrict__ lamq, double *lamb,
                                                                double *out_q, double *out_b) {
    int i, j, k;
    size_t p;
    if (!adj_cell(g, i, j, k, p)) return;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const double s = 1.0 / 16.0;
    const double *Lx = lamBc, *Ly = lamBc + n, *Lz = lamBc + 2 * n;
    const double bx = (9.0 * (Lx[g.at(i + 1, j, k)] + Lx[p]) - (Lx[g.at(i + 2, j, k)] + Lx[g.at(i - 1, j, k)])) * s;
    const double by = (9.0 * (Ly[g.at(i, j + 1, k)] + Ly[p]) - (Ly[g.at(i, j + 2, k)] + Ly[g.at(i, j - 1, k)])) * s;
    const double bz = (9.0 * (Lz[g.at(i, j, k + 1)] + Lz[p]) - (Lz[g.at(i, j, k + 2)] + Lz[g.at(i, j, k - 1)])) * s;
    const double bb[3] = {bx, by, bz};
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        lamb[(size_t)f * n + p] = bb[f];
        out_b[(size_t)f * n + p] += bb[f];
    }
#pragma unroll
    for (int f = 0; f < 5; ++f) out_q[(size_t)f * n + p] += lamq[(size_t)f * n + p];
}

// ---------------------------------------------------------------- misfit

// L = 1/2 dV sum over cells of |q - q*|^2 + |b - b*|^2 (five conserved and
// three face fields); lam = dV (q - q*), dV (b - b*).  Per-block partial sums.
static __global__ void __launch_bounds__(kRedThreads) misfit_partial_kernel(long long n, double dV, const double *q,
                                                                            const double *b, const double *tq,
                                                                            const double *tb, double *lq, double *lb,
                                                                            double *part) {
    __shared__ double red[32];
    double v[1] = {0.0};
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int f = 0; f < 5; ++f) {
            const size_t o = (size_t)f * (size_t)n + (size_t)p;
            const double d = q[o] - tq[o];
            v[0] += d * d;
            lq[o] = dV * d;
        }
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const size_t o = (size_t)f * (size_t)n + (size_t)p;
            const double d = b[o] - tb[o];
            v[0] += d * d;
            lb[o] = dV * d;
        }
    }
    bool ismax[1] = {false};
    block_reduce<double, 1>(v, ismax, red);
    if (threadIdx.x == 0) part[blockIdx.x] = 0.5 * dV * v[0];
}

// ---------------------------------------------------------------- initial state

// Face field b = curl A + B0 of an edge vector potential (A_x at (i, j+1/2,
// k+1/2), A_y at (i+1/2, j, k+1/2), A_z at (i+1/2, j+1/2, k) in cell units
// from the centre of cell (i, j, k)), first-order discrete curl (Sec. 4.1).
static __global__ void __launch_bounds__(256) ic_curl_kernel(AdjGrid g, const double *__restrict__ A, double B0x,
                                                             double B0y, double B0z, double *bface) {
    int i, j, k;
    size_t p;
    if (!adj_cell(g, i, j, k, p)) return;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const double *Ax = A, *Ay = A + n, *Az = A + 2 * n;
    bface[p] = (Az[p] - Az[g.at(i, j - 1, k)]) * g.rdy - (Ay[p] - Ay[g.at(i, j, k - 1)]) * g.rdz + B0x;
    bface[n + p] = (Ax[p] - Ax[g.at(i, j, k - 1)]) * g.rdz - (Az[p] - Az[g.at(i - 1, j, k)]) * g.rdx + B0y;
    bface[2 * n + p] = (Ay[p] - Ay[g.at(i - 1, j, k)]) * g.rdx - (Ax[p] - Ax[g.at(i, j - 1, k)]) * g.rdy + B0z;
}

// sixth-order face -> centre weights of the initial conditions (Sec. 4.14),
// faces i-5/2 .. i+5/2 = face indices i-3 .. i+2, divided by 256
__device__ __forceinline__ double ic_w6(int o) {
    return o == 0 || o == 5 ? 3.0 / 256.0 : o == 1 || o == 4 ? -25.0 / 256.0 : 150.0 / 256.0;
}

__device__ __forceinline__ void ic_cell_field(const AdjGrid &g, const double *bface, int i, int j, int k,
                                              double (&Bc)[3]) {
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    Bc[0] = Bc[1] = Bc[2] = 0.0;
#pragma unroll
    for (int o = 0; o < 6; ++o) {
        const double w = ic_w6(o);
        Bc[0] += w * bface[g.at(i - 3 + o, j, k)];
        Bc[1] += w * bface[n + g.at(i, j - 3 + o, k)];
        Bc[2] += w * bface[2 * n + g.at(i, j, k - 3 + o)];
    }
}

// conserved state (rho, rho v, E) with E from Eq. P, the cell field from the
// sixth-order interpolation of the faces
static __global__ void __launch_bounds__(256) ic_cons_kernel(AdjGrid g, double gm1, const double *__restrict__ rho,
                                                             const double *__restrict__ v, const double *__restrict__ P,
                                                             const double *__restrict__ bface, double *cons) {
    int i, j, k;
    size_t p;
    if (!adj_cell(g, i, j, k, p)) return;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    double Bc[3];
    ic_cell_field(g, bface, i, j, k, Bc);
    const double r = rho[p], vx = v[p], vy = v[n + p], vz = v[2 * n + p];
    cons[p] = r;
    cons[n + p] = r * vx;
    cons[2 * n + p] = r * vy;
    cons[3 * n + p] = r * vz;
    cons[4 * n + p] = P[p] / gm1 + 0.5 * r * (vx * vx + vy * vy + vz * vz) + 0.5 * (Bc[0] * Bc[0] + Bc[1] * Bc[1] + Bc[2] * Bc[2]);
}

// adjoint of ic_cons_kernel in rho and v; lamBc = Bc lamE (3 planes, scratch)
static __global__ void __launch_bounds__(256) ic_cons_adjoint_kernel(AdjGrid g, const double *__restrict__ rho,
                                                                     const double *__restrict__ v,
                                                                     const double *__restrict__ bface,
                                                                     const double *__restrict__ lcons, double *lrho,
                                                                     double *lv, double *lBc) {
    int i, j, k;
    size_t p;
    if (!adj_cell(g, i, j, k, p)) return;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    double Bc[3];
    ic_cell_field(g, bface, i, j, k, Bc);
    const double r = rho[p], vv[3] = {v[p], v[n + p], v[2 * n + p]};
    const double lE = lcons[4 * n + p];
    double lr = lcons[p] + 0.5 * lE * (vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2]);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double lm = lcons[(size_t)(1 + d) * n + p];
        lr += vv[d] * lm;
        lv[(size_t)d * n + p] = r * lm + r * vv[d] * lE;
        lBc[(size_t)d * n + p] = Bc[d] * lE;
    }
    lrho[p] = lr;
}

// lamb = lam_bface + (sixth-order interpolation)^T lamBc
static __global__ void __launch_bounds__(256) ic_interp_adjoint_kernel(AdjGrid g, const double *__restrict__ lbface,
                                                                       const double *__restrict__ lBc, double *lb) {
    int i, j, k;
    size_t p;
    if (!adj_cell(g, i, j, k, p)) return;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    double s[3] = {lbface[p], lbface[n + p], lbface[2 * n + p]};
    // face m feeds cell m + 3 - o with weight w_o
#pragma unroll
    for (int o = 0; o < 6; ++o) {
        const double w = ic_w6(o);
        s[0] += w * lBc[g.at(i + 3 - o, j, k)];
        s[1] += w * lBc[n + g.at(i, j + 3 - o, k)];
        s[2] += w * lBc[2 * n + g.at(i, j, k + 3 - o)];
    }
    lb[p] = s[0];
    lb[n + p] = s[1];
    lb[2 * n + p] = s[2];
}

// lamA = curl^T lamb (transpose of ic_curl_kernel)
static __global__ void __launch_bounds__(256) ic_curl_adjoint_kernel(AdjGrid g, const double *__restrict__ lb,
                                                                     double *lA) {
    int i, j, k;
    size_t p;
    if (!adj_cell(g, i, j, k, p)) return;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const double *bx = lb, *by = lb + n, *bz = lb + 2 * n;
    // b_y(i,j,k) has +A_x/dz, b_y(i,j,k+1) -A_x/dz; b_z(i,j,k) -A_x/dy, b_z(i,j+1,k) +A_x/dy
    lA[p] = (by[p] - by[g.at(i, j, k + 1)]) * g.rdz - (bz[p] - bz[g.at(i, j + 1, k)]) * g.rdy;
    // b_z: +A_y/dx at (i), -A_y/dx at (i+1); b_x: -A_y/dz at (k), +A_y/dz at (k+1)
    lA[n + p] = (bz[p] - bz[g.at(i + 1, j, k)]) * g.rdx - (bx[p] - bx[g.at(i, j, k + 1)]) * g.rdz;
    // b_x: +A_z/dy at (j), -A_z/dy at (j+1); b_y: -A_z/dx at (i), +A_z/dx at (i+1)
    lA[2 * n + p] = (bx[p] - bx[g.at(i, j + 1, k)]) * g.rdy - (by[p] - by[g.at(i + 1, j, k)]) * g.rdx;
}

// Defined in w5ct_adjoint{32,64}{js,z}.cu (one translation unit per
// arithmetic type and WENO variant, compiled in parallel).
template <typename B, int VAR>
cudaError_t launch_adj_sweep(int axis, const AdjSweepArgs<B> &a, cudaStream_t s);

template <typename B, int VAR>
cudaError_t launch_adj_sweep_impl(int axis, const AdjSweepArgs<B> &a, cudaStream_t s) {
    const long long n = (long long)a.nx * a.ny * a.nz;
    const unsigned nb = (unsigned)((n + 127) / 128);
    if (axis == 0)
        adj_face_kernel<0, B, VAR><<<nb, 128, 0, s>>>(a);
    else if (axis == 1)
        adj_face_kernel<1, B, VAR><<<nb, 128, 0, s>>>(a);
    else
        adj_face_kernel<2, B, VAR><<<nb, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace w5ct
