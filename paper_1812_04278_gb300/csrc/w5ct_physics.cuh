// w5ct_physics.cuh -- device arithmetic of the WENO5 + CT ideal-MHD scheme
// of Donnert et al. (arXiv:1812.04278), templated on the arithmetic type
// (double for the FP64 path, float for the FP32-bulk path).
//
//   cell_fill  : primitives (Eq. P), flux along the sweep axis (Eq. fluxes),
//                wave speeds (Eqs. slow, fast, ca) of one cell.
//   face_flux  : characteristic WENO5 / WENO5-Z flux at one interface
//                (Sec. 2.2, Eq. FWENO) with the eigenvectors of Appendix A.
//
// Readings of the garbled passages (identical in the CPU oracle):
//   P* = P + B^2/2; fast/slow speeds from the discriminant
//   d = (c_s^2 - c_A^2)^2 + b_t^2 (b_t^2 + 2 c_A^2 + 2 c_s^2) without
//   cancellation, c_slow^2 = c_s^2 c_A^2 / c_f^2; Appendix A's "slow" block is
//   the Alfven pair (m = 2, 6) and its "Alfven" block the slow pair (m = 3, 5);
//   upper signs for m <= 3; beta normalised by |B_t|; sgn(B_n) = +1 iff
//   B_n >= eps_B; fast-mode left eigenvector with the 1/(2 c_s^2) factor on
//   every component, gamma_1 alpha_f v^2 +- Gamma_f, -+ alpha_f c_f and
//   + sqrt(rho) c_s alpha_s beta in the field rows; entropy right eigenvector
//   energy row v^2/2; interface state = mean of the two cells' primitives;
//   alpha(m) = max(|lambda_m(i)|, |lambda_m(i+1)|); WENO-Z weights
//   d_k (1 + (tau_5/(eps_Z + IS_k))^2).
#pragma once
#include <cuda_runtime.h>
#include <type_traits>

namespace w5ct {

// per-cell quantities kept in shared memory during a sweep (frame components)
enum CellQ {
    C_RHO = 0, C_VN, C_VT1, C_VT2, C_BN, C_BT1, C_BT2, C_P,   // primitives w
    C_RHOQ, C_MN, C_MT1, C_MT2, C_E,                          // conserved u (rho, m, E)
    C_F0, C_F1, C_F2, C_F3, C_F4, C_F5, C_F6,                 // flux along n
    C_CF, C_CA, C_CSL,                                        // c_fast, c_Alfven, c_slow
    NCQ
};

// The FP64 sweep's cell box holds, after its difference pass, besides the
// NCQ quantities of cell_fill_frame: the forward differences dF_c(i) =
// F_c(i+1) - F_c(i) of the seven frame fluxes (planes C_DF0..C_DF6) and
// du_c(i) = u_c(i+1) - u_c(i) of the conserved 7-vector -- in place of u_c
// for rho, m and E (planes C_RHOQ, C_MN, C_MT1, C_MT2, C_E), in C_DU4, C_DU5
// for B_t1, B_t2 (whose planes stay the primitives).
enum BoxQ { C_DF0 = NCQ, C_DU4 = NCQ + 7, C_DU5, NBQ };

// The difference pass pays in double, where the sweep is bound by the FP64
// pipe and it removes 77 FP64 operations per interface (the stencil
// differences and the central combination) for 14 per cell; in float its
// extra barriers and shared-memory traffic cost more than the FP32
// operations it saves.  Boxes of the compile-time tiles (sweep_tile_at):
template <typename Real>
__host__ __device__ constexpr bool box_diff() {
    return sizeof(Real) == 8;
}
template <typename Real>
__host__ __device__ constexpr int box_quantities() {
    return box_diff<Real>() ? NBQ : NCQ;
}

template <typename Real>
struct Phys {
    Real gamma, gm1, g1, g2;     // gamma, gamma-1, (gamma-1)/2, (gamma-2)/(gamma-1)
    Real eps_w;                  // WENO epsilon (JS or Z, per the variant)
    Real eps_b;                  // eps_B of Appendix A
    Real eps_b2;                 // threshold on c_f^2 - c_slow^2 (eps_B^2, >= FLT_MIN in float)
    Real rho_min, p_min;
    // lower bound on c_s^2 in the interface eigenvectors, relative to
    // v^2 + c_A^2 + b_t^2 (0 in double; see face_flux)
    Real cs2_rel;
    int floors;
};

// float_based<Real> selects the float-specific guards of the FP32-bulk
// arithmetic.
template <typename R>
constexpr bool float_based = std::is_same<R, float>::value;

// ---------------------------------------------------------------- math helpers
template <typename Real> struct M;
// Reciprocal of a positive finite double by Newton-Raphson iteration on
// f(r) = 1/r - y (r' = r + r (1 - y r), quadratic convergence), started from
// the hardware's approximate reciprocal (PTX rcp.approx.ftz.f64); two
// iterations reach the rounding limit.  The FP64 sweep is bound by the FP64
// pipe, and this takes fewer of its instructions than the IEEE division.
// Only for y > 0 finite and normal (the callers guard zero; a reciprocal below
// the normal range is flushed to zero).
__device__ __forceinline__ double drcp_newton(double y) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(y));
    double e = fma(-y, r, 1.0);
    r = fma(r, e, r);
    e = fma(-y, r, 1.0);
    return fma(r, e, r);
}

template <> struct M<double> {
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double div_(double a, double b) { return a * drcp_newton(b); }
    static __device__ __forceinline__ double rcp_(double x) { return drcp_newton(x); }
    static __device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
    static __device__ __forceinline__ double abs_(double x) { return fabs(x); }
    static __device__ __forceinline__ double max_(double a, double b) { return fmax(a, b); }
    static __device__ __forceinline__ double min_(double a, double b) { return fmin(a, b); }
    static __device__ __forceinline__ bool finite_pos(double x) { return x > 0.0 && x < 1.0e308; }
};
template <> struct M<float> {
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float div_(float a, float b) { return __fdividef(a, b); }
    static __device__ __forceinline__ float rcp_(float x) { return __fdividef(1.0f, x); }
    static __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float abs_(float x) { return fabsf(x); }
    static __device__ __forceinline__ float max_(float a, float b) { return fmaxf(a, b); }
    static __device__ __forceinline__ float min_(float a, float b) { return fminf(a, b); }
    static __device__ __forceinline__ bool finite_pos(float x) { return x > 0.0f && x < 3.0e38f; }
};

// ---------------------------------------------------------------- wave speeds
// c_f^2 - c_s^2 (fmc), c_s^2 - c_slow^2 (cms) without cancellation, and c_f^2.
// The larger of the two differences is (sd + |aa|) / 2 (aa = c_A^2 + b_t^2 -
// c_s^2), the other c_s^2 b_t^2 over it.  In float the two cases are formed
// without branches (0.5% faster sweep), in double with them (0.5% faster
// there); the results are the same bits.
template <typename Real>
__device__ __forceinline__ void speeds_fast(Real cs2, Real ca2, Real bt2, Real &fmc, Real &cms, Real &cf2) {
    using m = M<Real>;
    const Real dd = (cs2 - ca2) * (cs2 - ca2) + bt2 * (bt2 + Real(2) * ca2 + Real(2) * cs2);
    const Real sd = m::sqrt_(dd);
    const Real aa = ca2 + bt2 - cs2;
    if constexpr (float_based<Real>) {
        const Real big = Real(0.5) * (sd + m::abs_(aa));
        const Real oth = big > Real(0) ? m::div_(cs2 * bt2, big) : Real(0);
        const bool fast_big = aa >= Real(0);
        fmc = fast_big ? big : oth;
        cms = fast_big ? oth : big;
    } else {
        if (aa >= Real(0)) {
            fmc = Real(0.5) * (aa + sd);
            cms = fmc > Real(0) ? m::div_(cs2 * bt2, fmc) : Real(0);
        } else {
            cms = Real(0.5) * (sd - aa);
            fmc = cms > Real(0) ? m::div_(cs2 * bt2, cms) : Real(0);
        }
    }
    cf2 = cs2 + fmc;
}

// speeds_fast and c_slow^2 = c_s^2 c_A^2 / c_f^2.
template <typename Real>
__device__ __forceinline__ void speeds(Real cs2, Real ca2, Real bt2, Real &fmc, Real &cms, Real &cf2, Real &csl2) {
    speeds_fast<Real>(cs2, ca2, bt2, fmc, cms, cf2);
    csl2 = cf2 > Real(0) ? M<Real>::div_(cs2 * ca2, cf2) : Real(0);
}

// ---------------------------------------------------------------- one cell
// Fills the NCQ per-cell quantities of a cell from its state in the sweep
// frame (n, t1, t2): momentum (mn, m1, m2), cell field (Bn, B1, B2).  sm
// points at the cell's slot of quantity 0; quantities are `stride` elements
// apart.
template <typename Real>
__device__ __forceinline__ void cell_fill_frame(Real *sm, int stride, Real rho, Real mn, Real m1, Real m2, Real E,
                                                Real Bn, Real B1, Real B2, const Phys<Real> &K, bool &bad, bool &hit) {
    using m = M<Real>;
    Real r = rho;
    if (K.floors && r < K.rho_min) { r = K.rho_min; hit = true; }
    const Real ir = m::rcp_(r);
    const Real vn = mn * ir, v1 = m1 * ir, v2 = m2 * ir;
    const Real vv = vn * vn + v1 * v1 + v2 * v2;
    const Real BB = Bn * Bn + B1 * B1 + B2 * B2;
    Real P = K.gm1 * (E - Real(0.5) * r * vv - Real(0.5) * BB);
    if (K.floors && P < K.p_min) { P = K.p_min; hit = true; }
    if (!(r > Real(0)) || !m::finite_pos(P)) bad = true;
    const Real Pt = P + Real(0.5) * BB;
    const Real vB = vn * Bn + v1 * B1 + v2 * B2;
    sm[C_RHO * stride] = r;
    sm[C_VN * stride] = vn;
    sm[C_VT1 * stride] = v1;
    sm[C_VT2 * stride] = v2;
    sm[C_BN * stride] = Bn;
    sm[C_BT1 * stride] = B1;
    sm[C_BT2 * stride] = B2;
    sm[C_P * stride] = P;
    sm[C_RHOQ * stride] = rho;
    sm[C_MN * stride] = mn;
    sm[C_MT1 * stride] = m1;
    sm[C_MT2 * stride] = m2;
    sm[C_E * stride] = E;
    // rho v_n = m_n (v = m / rho with the same, possibly floored, rho)
    sm[C_F0 * stride] = mn;
    sm[C_F1 * stride] = mn * vn + Pt - Bn * Bn;
    sm[C_F2 * stride] = mn * v1 - Bn * B1;
    sm[C_F3 * stride] = mn * v2 - Bn * B2;
    sm[C_F4 * stride] = B1 * vn - Bn * v1;
    sm[C_F5 * stride] = B2 * vn - Bn * v2;
    sm[C_F6 * stride] = (E + Pt) * vn - Bn * vB;
    const Real cs2 = K.gamma * P * ir;
    const Real ca2 = Bn * Bn * ir;
    const Real bt2 = (B1 * B1 + B2 * B2) * ir;
    Real fmc, cms, cf2, csl2;
    speeds<Real>(cs2, ca2, bt2, fmc, cms, cf2, csl2);
    sm[C_CF * stride] = m::sqrt_(cf2);
    sm[C_CA * stride] = m::abs_(Bn) * m::rsqrt_(r);     // |B_n| / sqrt(rho)
    sm[C_CSL * stride] = m::sqrt_(csl2);
}

// cell_fill_frame for a sweep along axis AX (frame (n, t1, t2) = (AX, AX+1,
// AX+2) mod 3) from the lab components
template <typename Real, int AX>
__device__ __forceinline__ void cell_fill(Real *sm, int stride, Real rho, Real mx, Real my, Real mz, Real E,
                                          Real Bx, Real By, Real Bz, const Phys<Real> &K, bool &bad, bool &hit) {
    constexpr int n = AX, t1 = (AX + 1) % 3, t2 = (AX + 2) % 3;
    const Real mm[3] = {mx, my, mz};
    const Real BB3[3] = {Bx, By, Bz};
    cell_fill_frame<Real>(sm, stride, rho, mm[n], mm[t1], mm[t2], E, BB3[n], BB3[t1], BB3[t2], K, bad, hit);
}

// the same with the axis known only at run time (selects, no indexed arrays)
template <typename Real>
__device__ __forceinline__ void cell_fill_axis(Real *sm, int stride, Real rho, Real mx, Real my, Real mz, Real E,
                                               Real Bx, Real By, Real Bz, int ax, const Phys<Real> &K, bool &bad,
                                               bool &hit) {
    const Real mn = ax == 0 ? mx : (ax == 1 ? my : mz);
    const Real m1 = ax == 0 ? my : (ax == 1 ? mz : mx);
    const Real m2 = ax == 0 ? mz : (ax == 1 ? mx : my);
    const Real Bn = ax == 0 ? Bx : (ax == 1 ? By : Bz);
    const Real B1 = ax == 0 ? By : (ax == 1 ? Bz : Bx);
    const Real B2 = ax == 0 ? Bz : (ax == 1 ? Bx : By);
    cell_fill_frame<Real>(sm, stride, rho, mn, m1, m2, E, Bn, B1, B2, K, bad, hit);
}

// The difference pass of a sweep's cell box, in two steps around a barrier
// (du overwrites u in place): box_diff_load reads the flux and conserved
// 7-vectors of cell i and of its successor i + st along the sweep axis and
// forms their differences; box_diff_store writes them.  sm points at the
// box, `stride` elements between quantities.
template <typename Real>
struct CellDiff {
    Real dF[7], dU[7];
};

template <typename Real>
__device__ __forceinline__ void box_diff_load(const Real *sm, int stride, int i, int st, CellDiff<Real> &d) {
    const Real *a = sm + i, *b = sm + i + st;
#pragma unroll
    for (int c = 0; c < 7; ++c) d.dF[c] = b[(C_F0 + c) * stride] - a[(C_F0 + c) * stride];
    constexpr int qU[7] = {C_RHOQ, C_MN, C_MT1, C_MT2, C_BT1, C_BT2, C_E};
#pragma unroll
    for (int c = 0; c < 7; ++c) d.dU[c] = b[qU[c] * stride] - a[qU[c] * stride];
}

template <typename Real>
__device__ __forceinline__ void box_diff_store(Real *sm, int stride, int i, const CellDiff<Real> &d) {
    Real *a = sm + i;
#pragma unroll
    for (int c = 0; c < 7; ++c) a[(C_DF0 + c) * stride] = d.dF[c];
    constexpr int qD[7] = {C_RHOQ, C_MN, C_MT1, C_MT2, C_DU4, C_DU5, C_E};
#pragma unroll
    for (int c = 0; c < 7; ++c) a[qD[c] * stride] = d.dU[c];
}

// fast signal speed |v_d| + c_f^d of a cell along axis d (Eq. cfl)
template <typename Real>
__device__ __forceinline__ Real signal_speed(Real r, Real vn, Real P, Real Bn, Real B1, Real B2, const Phys<Real> &K) {
    using m = M<Real>;
    const Real ir = m::rcp_(r);
    const Real cs2 = K.gamma * P * ir;
    const Real ca2 = Bn * Bn * ir;
    const Real bt2 = (B1 * B1 + B2 * B2) * ir;
    Real fmc, cms, cf2, csl2;
    speeds<Real>(cs2, ca2, bt2, fmc, cms, cf2, csl2);
    return m::abs_(vn) + m::sqrt_(cf2);
}

// ---------------------------------------------------------------- WENO
// phi_N(a, b, c, d) of Sec. 2.2 with JS (VAR = 0) or WENO-Z (VAR = 1)
// weights, in the form the kernels evaluate.
//
// Two rewrites that leave phi_N unchanged up to rounding:
// * the weights depend only on the ratios of eps + IS_k (JS: alpha_k =
//   d_k / (eps + IS_k)^2 normalised; WENO-Z: tau_5 / (eps + IS_k)), so the
//   smoothness indicators are evaluated as IS_k / 3 = (13/3) x^2 + y^2 with
//   eps / 3 (the caller passes it);
// * with w_k = a_k / D (D = a_0 + a_1 + a_2) and the second differences
//   t1 = a - 2b + c = x0 - y0, t2 = b - 2c + d = y0 - z0 of the first ones
//   (x0 = a - b, y0 = b - c, z0 = c - d, also those of the indicators),
//   phi_N = w_0 t1 / 3 + (w_2 - 1/2) t2 / 6
//         = [a_0 t1 + (a_2 / 2 - D / 4) t2] / (3 D);
//   in double each interpolant returns that numerator and D, and weno_field
//   divides once for the two; in float the weights are normalised first
//   (D = 1) and phi_N = Nn / 3.
//
// smoothness3 returns s_k = eps/3 + IS_k/3, the epsilon added inside the
// last FMA of each indicator, and the first differences x0, y0, z0.
template <typename Real>
__device__ __forceinline__ void smoothness3(Real a, Real b, Real c, Real d, Real eps3, Real &s0, Real &s1, Real &s2,
                                            Real &x0, Real &y0, Real &z0) {
    const Real k = Real(13.0 / 3.0);
    x0 = a - b;
    const Real x1 = a - Real(3) * b;
    s0 = (k * x0) * x0 + (x1 * x1 + eps3);
    y0 = b - c;
    const Real y1 = b + c;
    s1 = (k * y0) * y0 + (y1 * y1 + eps3);
    z0 = c - d;
    const Real z1 = Real(3) * c - d;
    s2 = (k * z0) * z0 + (z1 * z1 + eps3);
}

// float: phi_N = Nn / 3 with the weights normalised here by one reciprocal
// (the WENO-Z ratio tau_5 / (eps + IS_k) is clamped at 1e18, so nothing
// overflows; unnormalised WENO-Z weights reach 1e36 in float)
template <int VAR>
__device__ __forceinline__ float phi_nf(float a, float b, float c, float d, float eps3) {
    float s0, s1, s2, x0, y0, z0;
    smoothness3<float>(a, b, c, d, eps3, s0, s1, s2, x0, y0, z0);
    float e0, e1, e2;   // alpha_k / d_k
    if constexpr (VAR == 0) {
        e0 = __fdividef(1.0f, s0 * s0);
        e1 = __fdividef(1.0f, s1 * s1);
        e2 = __fdividef(1.0f, s2 * s2);
    } else {
        const float tau = fabsf(s0 - s2);   // |IS_0 - IS_2| / 3
        const float r0 = fminf(tau * __fdividef(1.0f, s0), 1.0e18f);
        const float r1 = fminf(tau * __fdividef(1.0f, s1), 1.0e18f);
        const float r2 = fminf(tau * __fdividef(1.0f, s2), 1.0e18f);
        e0 = __fmaf_rn(r0, r0, 1.0f);
        e1 = __fmaf_rn(r1, r1, 1.0f);
        e2 = __fmaf_rn(r2, r2, 1.0f);
    }
    // D = e0 + 6 e1 + 3 e2; a_2 / 2 = 1.5 e2
    const float inv = __fdividef(1.0f, __fmaf_rn(3.0f, e2, __fmaf_rn(6.0f, e1, e0)));
    return (e0 * inv) * (x0 - y0) + __fmaf_rn(e2, 1.5f * inv, -0.25f) * (y0 - z0);
}

// double: the weights times the common factor (s_0 s_1 s_2)^2, so that no
// weight needs a division; phi_N = Nn / (3 D), and the two interpolants of
// one field share a single division in weno_field.  The linear weights
// d = (1, 6, 3) enter the sum and the numerator by FMAs.
template <int VAR>
__device__ __forceinline__ void phi_nd(double a, double b, double c, double d, double eps3, double &Nn, double &Dn) {
    double s0, s1, s2, x0, y0, z0;
    smoothness3<double>(a, b, c, d, eps3, s0, s1, s2, x0, y0, z0);
    double W0, V1, V2;   // alpha_k / d_k times the common factor
    if constexpr (VAR == 0) {
        // alpha_k = d_k / s_k^2 times (s0 s1 s2)^2
        const double p0 = s1 * s2, p1 = s0 * s2, p2 = s0 * s1;
        W0 = p0 * p0;
        V1 = p1 * p1;
        V2 = p2 * p2;
    } else {
        // alpha_k = d_k (1 + tau^2 / s_k^2) times (s0 s1 s2)^2: with e_k =
        // s_k^2 and E = e0 e1 e2, (e_k + tau^2) prod_{j != k} e_j = E + tau^2
        // prod_{j != k} e_j, one FMA per weight
        const double tau = fabs(s0 - s2);   // |IS_0 - IS_2| / 3
        const double tt = tau * tau;
        const double e0 = s0 * s0, e1 = s1 * s1, e2 = s2 * s2;
        const double e12 = e1 * e2, e02 = e0 * e2, e01 = e0 * e1;
        const double E = e0 * e12;
        W0 = fma(tt, e12, E);
        V1 = fma(tt, e02, E);
        V2 = fma(tt, e01, E);
    }
    Dn = fma(3.0, V2, fma(6.0, V1, W0));
    // a_0 t1 + (a_2 / 2 - D / 4) t2 with a_2 = 3 V2
    Nn = W0 * (x0 - y0) + fma(1.5, V2, -0.25 * Dn) * (y0 - z0);
}

// ---------------------------------------------------------------- double-word
// A double-word number is the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi) / 2: 48 significand bits (unit roundoff u^2, u = 2^-24)
// and float's exponent range.  Each operation is a short sequence of FP32
// operations built on the error-free transforms TwoSum (Knuth), Fast2Sum
// (Dekker; |a| >= |b|) and TwoProd (one FMA), as analysed by Joldes, Muller
// and Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic", ACM TOMS 44(2), 2017.  The intrinsics keep every
// step a separately rounded operation (no contraction into FMAs).
struct dw {
    float hi, lo;
};

__device__ __forceinline__ dw ef_fast2sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dw ef_twosum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    return {s, __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv))};
}
__device__ __forceinline__ dw ef_twoprod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
// x + y: TwoSum of the high parts, the low parts added to its error term,
// Fast2Sum (the "sloppy" sum of Joldes et al.).  The error is about
// 2 u^2 (|x| + |y|): relative to the result for operands of one sign, and
// relative to the operands where they cancel -- the accuracy the WENO
// differences need, whose double inputs enter with relative errors of
// 2^-49 from the conversion anyway.
__device__ __forceinline__ dw dw_add(dw x, dw y) {
    const dw s = ef_twosum(x.hi, y.hi);
    return ef_fast2sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dw dw_neg(dw x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dw dw_sub(dw x, dw y) { return dw_add(x, dw_neg(y)); }
// x * y with y a float, and with y a double-word
__device__ __forceinline__ dw dw_mul_f(dw x, float y) {
    const dw c = ef_twoprod(x.hi, y);
    return ef_fast2sum(c.hi, __fmaf_rn(x.lo, y, c.lo));
}
__device__ __forceinline__ dw dw_mul(dw x, dw y) {
    const dw c = ef_twoprod(x.hi, y.hi);
    const float t = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.hi));
    return ef_fast2sum(c.hi, __fadd_rn(c.lo, t));
}
// x / y: the float quotient q from a reciprocal refined by one Newton step,
// the residual x - y q in double-word, and its quotient as the correction
__device__ __forceinline__ dw dw_div(dw x, dw y) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y.hi));
    r = __fmaf_rn(r, __fmaf_rn(-y.hi, r, 1.0f), r);
    const float q = __fmul_rn(x.hi, r);
    const dw yq = dw_mul_f(y, q);
    const dw p = ef_twosum(x.hi, -yq.hi);
    const float d = __fadd_rn(p.hi, __fadd_rn(__fsub_rn(p.lo, yq.lo), x.lo));
    return ef_fast2sum(q, __fmul_rn(d, r));
}
__device__ __forceinline__ bool dw_eq(dw x, dw y) { return x.hi == y.hi && x.lo == y.lo; }

// A double as a double-word on the integer pipes (IEEE 754 binary64 layout:
// exponent bias 1023, 52 fraction bits): hi is x truncated to 24 significand
// bits, lo the remaining 29 bits rounded to 24, then renormalised (Fast2Sum).
// |x| below 2^-126 gives 0, |x| at or above 2^128 gives +-inf: neither
// occurs for the WENO inputs of a physical state, whose relative precision
// here is 2^-48.
__device__ __forceinline__ dw dw_from_double(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned hw = (unsigned)(u >> 32), lw = (unsigned)u;
    const unsigned sgn = hw & 0x80000000u;
    const int e = (int)((hw >> 20) & 0x7ffu);
    const unsigned hb = sgn | ((unsigned)(e - 896) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29);
    const float m = __uint2float_rn(lw & 0x1fffffffu);
    const float lo = __fmul_rn(m, __uint_as_float((unsigned)(e - 948) << 23));   // m 2^(e - 1075)
    float h = __uint_as_float(hb), l = __uint_as_float(__float_as_uint(lo) | sgn);
    if (e <= 948) l = 0.0f;
    if (e <= 896) h = 0.0f;
    if (e >= 1151) {
        h = __uint_as_float(sgn | 0x7f800000u);
        l = 0.0f;
    }
    return ef_fast2sum(h, l);
}

// A float as the double of equal value on the integer pipes (binary32:
// bias 127, 23 fraction bits); zeros and subnormals give 0, infinities and
// NaNs a NaN.
__device__ __forceinline__ double dw_f2d(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned ef = (b >> 23) & 0xffu;
    const unsigned hw = (b & 0x80000000u) | ((ef + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    double d = __hiloint2double((int)hw, (int)(b << 29));
    if (ef == 0u) d = 0.0;
    if (ef == 0xffu) d = __longlong_as_double(0x7ff8000000000000LL);
    return d;
}

// phi_N (Sec. 2.2) of four double-word stencil differences (eps3 as in
// smoothness3), returned as 3 phi_N = (e_0 / D) t1 + (3 e_2 / (2 D) - 1/4) t2
// with e_k = alpha_k / d_k up to a common factor and D = e_0 + 6 e_1 + 3 e_2.
// The weights are formed relative to the smallest s_k (index m), so that no
// intermediate leaves float's range: with rho_k = s_m / s_k (rho_m = 1),
//   JS: alpha_k / d_k = 1 / s_k^2 = rho_k^2 / s_m^2, the common factor dropped;
//   Z:  alpha_k / d_k = 1 + (tau / s_k)^2 = 1 + (R rho_k)^2 with R = tau / s_m,
//       and, where R > 1e18, R^2 rho_k^2 (the 1 is below 1e-36 of the rest).
// Where eps / 3 is below float's range (WENO-Z) an indicator of a stencil
// without variation is 0; then rho_k = 0 for the others (their weights
// vanish against it, as in double), rho_k = 1 between equal indicators, and
// R = 0 where tau = 0.  An indicator below float's normal range (stencil
// differences under about 1e-19) counts as 0 as well: the reciprocal of a
// subnormal is not representable, and in double the weights of such
// stencils are set by rounding noise anyway.
template <int VAR>
__device__ __forceinline__ dw phi_dw(dw a, dw b, dw c, dw d, dw eps3) {
    const dw x0 = dw_sub(a, b), y0 = dw_sub(b, c), z0 = dw_sub(c, d);
    const dw x1 = dw_sub(x0, dw{2.0f * b.hi, 2.0f * b.lo});     // a - 3b
    const dw y1 = dw_add(b, c);
    const dw z1 = dw_add(z0, dw{2.0f * c.hi, 2.0f * c.lo});     // 3c - d
    const dw k = {4.33333349f, -1.58945719e-07f};              // 13/3
    auto normal_or_zero = [](dw s) { return s.hi < 1.17549435e-38f ? dw{0.0f, 0.0f} : s; };
    const dw s0 = normal_or_zero(dw_add(dw_add(dw_mul(k, dw_mul(x0, x0)), dw_mul(x1, x1)), eps3));
    const dw s1 = normal_or_zero(dw_add(dw_add(dw_mul(k, dw_mul(y0, y0)), dw_mul(y1, y1)), eps3));
    const dw s2 = normal_or_zero(dw_add(dw_add(dw_mul(k, dw_mul(z0, z0)), dw_mul(z1, z1)), eps3));
    dw sm = s0;
    if (s1.hi < sm.hi) sm = s1;
    if (s2.hi < sm.hi) sm = s2;
    const dw one = {1.0f, 0.0f};
    const dw r0 = dw_eq(s0, sm) ? one : dw_div(sm, s0);
    const dw r1 = dw_eq(s1, sm) ? one : dw_div(sm, s1);
    const dw r2 = dw_eq(s2, sm) ? one : dw_div(sm, s2);
    dw e0 = dw_mul(r0, r0), e1 = dw_mul(r1, r1), e2 = dw_mul(r2, r2);
    if constexpr (VAR == 1) {
        dw tau = dw_sub(s0, s2);
        if (tau.hi < 0.0f) tau = dw_neg(tau);
        const dw R = tau.hi == 0.0f ? dw{0.0f, 0.0f} : dw_div(tau, sm);
        if (R.hi <= 1.0e18f) {
            const dw R2 = dw_mul(R, R);
            e0 = dw_add(one, dw_mul(R2, e0));
            e1 = dw_add(one, dw_mul(R2, e1));
            e2 = dw_add(one, dw_mul(R2, e2));
        }
    }
    const dw D = dw_add(dw_add(e0, dw_mul_f(e1, 6.0f)), dw_mul_f(e2, 3.0f));
    const dw inv = dw_div(one, D);
    const dw w0 = dw_mul(e0, inv);
    const dw w2 = dw_add(dw_mul_f(dw_mul(e2, inv), 1.5f), dw{-0.25f, 0.0f});
    return dw_add(dw_mul(w0, dw_sub(x0, y0)), dw_mul(w2, dw_sub(y0, z0)));
}

// Eq. (FWENO) for one characteristic field from its 11 projections:
// P[0] = L.central, P[1..5] = L.dF at i-3/2 .. i+5/2, P[6..10] = L.du there.
//
// The split differences are (dF +- alpha dq)/2.  IS_k scales with the square
// of its arguments and phi_N linearly, so phi_N(x/2; eps) = phi_N(x; 4 eps)/2
// for both weight variants: the factor 1/2 is applied once to the result.
// With the IS_k / 3 form above the epsilon passed in is eps43 = 4 eps / 3,
// and F = P[0] + (phi_N^- - phi_N^+)/2 = P[0] + (Nm/Dm - Np/Dp)/6.
//
// DWW (double only): the split differences, formed in double, go to
// double-word, phi_dw evaluates both interpolants there, and their
// difference returns to double for the last FMAs with P[0].
template <typename Real, int VAR, bool DWW = false>
__device__ __forceinline__ Real weno_field(const Real P[11], Real alpha, Real eps43) {
    Real p[5], q[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        p[j] = P[1 + j] + alpha * P[6 + j];
        q[j] = P[1 + j] - alpha * P[6 + j];
    }
    if constexpr (std::is_same<Real, double>::value && DWW) {
        dw pd[5], qd[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            pd[j] = dw_from_double(p[j]);
            qd[j] = dw_from_double(q[j]);
        }
        const dw e3 = dw_from_double(eps43);
        const dw Np = phi_dw<VAR>(pd[0], pd[1], pd[2], pd[3], e3);
        const dw Nm = phi_dw<VAR>(qd[4], qd[3], qd[2], qd[1], e3);
        const dw r = dw_sub(Nm, Np);
        return fma(1.0 / 6.0, dw_f2d(r.hi), fma(1.0 / 6.0, dw_f2d(r.lo), P[0]));
    }
    if constexpr (std::is_same<Real, double>::value) {
        double Np, Dp, Nm, Dm;
        phi_nd<VAR>(p[0], p[1], p[2], p[3], eps43, Np, Dp);
        phi_nd<VAR>(q[4], q[3], q[2], q[1], eps43, Nm, Dm);
        const double prod = Dp * Dm;
        if (prod > 1e-290 && prod < 1e290) {
            // -Np/Dp + Nm/Dm over the common denominator: one reciprocal
            return P[0] + (1.0 / 6.0) * ((Nm * Dp - Np * Dm) * drcp_newton(prod));
        }
        return P[0] + (1.0 / 6.0) * (Nm / Dm - Np / Dp);
    } else {
        static_assert(std::is_same<Real, float>::value, "weno_field takes float or double");
        const float Np = phi_nf<VAR>(p[0], p[1], p[2], p[3], eps43);
        const float Nm = phi_nf<VAR>(q[4], q[3], q[2], q[1], eps43);
        return __fmaf_rn(1.0f / 6.0f, Nm - Np, P[0]);
    }
}

// ---------------------------------------------------------------- float
// In float the 11 stencil vectors are kept as the central one, X0, and the
// five pairs X2[j] = (dF_j, du_j) (vectors 1 + j and 6 + j), which share
// every projection coefficient: one packed two-lane FMA (sm_100 f32x2)
// projects both.  Each lane rounds exactly as the scalar FMA would.
__device__ __forceinline__ float2 bcast2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// P = sum_k L[k] X[ci[k]] for the 11 vectors (scalar central, packed pairs)
template <int N>
__device__ __forceinline__ void project_f(const float (&X0)[7], const float2 (&X2)[5][7], const int (&ci)[N],
                                          const float (&L)[N], float &P0, float2 (&P2)[5]) {
    float p = L[0] * X0[ci[0]];
#pragma unroll
    for (int k = 1; k < N; ++k) p = __fmaf_rn(L[k], X0[ci[k]], p);
    P0 = p;
    float2 Lb[N];
#pragma unroll
    for (int k = 0; k < N; ++k) Lb[k] = bcast2(L[k]);
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        float2 q = __fmul2_rn(Lb[0], X2[j][ci[0]]);
#pragma unroll
        for (int k = 1; k < N; ++k) q = __ffma2_rn(Lb[k], X2[j][ci[k]], q);
        P2[j] = q;
    }
}

// weno_field's 11 projections from the central value and the five pairs
__device__ __forceinline__ void unpack11(float P0, const float2 (&P2)[5], float (&P)[11]) {
    P[0] = P0;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        P[1 + j] = P2[j].x;
        P[6 + j] = P2[j].y;
    }
}

// (P_c + P_s, P_c - P_s) of a mode pair, both packed halves at once
__device__ __forceinline__ void split_pair_f(float Pc0, const float2 (&Pc2)[5], float Ps0, const float2 (&Ps2)[5],
                                             float (&Pu)[11], float (&Pl)[11]) {
    float2 U[5], D[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        U[j] = __fadd2_rn(Pc2[j], Ps2[j]);
        D[j] = __fadd2_rn(Pc2[j], neg2(Ps2[j]));
    }
    unpack11(Pc0 + Ps0, U, Pu);
    unpack11(Pc0 - Ps0, D, Pl);
}

// ---------------------------------------------------------------- one face
// Characteristic WENO flux at the face between stencil cells 2 and 3 of the
// six cells at sm + k*st (k = 0..5); quantities are `ncell` elements apart.
// Ff receives the frame flux (rho, m_n, m_t1, m_t2, B_t1, B_t2, E) and
// s1, s2 the CT transport fluxes F_{B_t} + <B_n v_t> of Eqs. (fct1)-(fct6).
template <typename Real, int VAR, bool DIFF = false, bool DWW = false>
__device__ __forceinline__ void face_flux(const Real *__restrict__ sm, int ncell, int st, const Phys<Real> &K,
                                          Real (&Ff)[7], Real &s1, Real &s2) {
    using m = M<Real>;
#define SMQ(q, k) sm[(q) * ncell + (k) * st]
    // physical central combination and differences (projection is linear)
    Real X[11][7];
#pragma unroll
    for (int c = 0; c < 7; ++c) {
        if constexpr (DIFF) {
            // from the box's forward differences (its difference pass):
            // X[1 + j] = dF(j), X[6 + j] = du(j), j = 0..4, and the central
            // combination (7 (f2 + f3) - (f1 + f4)) / 12 written as
            // f2 + (6 dF(2) + dF(1) - dF(3)) / 12
            const int qD = C_DF0 + c;
            const int qU = c == 0 ? C_RHOQ : c == 1 ? C_MN : c == 2 ? C_MT1 : c == 3 ? C_MT2 : c == 4 ? C_DU4
                           : c == 5 ? C_DU5 : C_E;
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                X[1 + j][c] = SMQ(qD, j);
                X[6 + j][c] = SMQ(qU, j);
            }
            X[0][c] = SMQ(C_F0 + c, 2) + (Real(6) * X[3][c] + X[2][c] - X[4][c]) * Real(1.0 / 12.0);
        } else {
            const int qF = C_F0 + c;
            const Real f0 = SMQ(qF, 0), f1 = SMQ(qF, 1), f2 = SMQ(qF, 2), f3 = SMQ(qF, 3), f4 = SMQ(qF, 4),
                       f5 = SMQ(qF, 5);
            X[1][c] = f1 - f0;
            X[2][c] = f2 - f1;
            X[3][c] = f3 - f2;
            X[4][c] = f4 - f3;
            X[5][c] = f5 - f4;
            // (7 (f2 + f3) - (f1 + f4)) / 12 from the differences
            X[0][c] = f2 + (Real(6) * X[3][c] + X[2][c] - X[4][c]) * Real(1.0 / 12.0);
            const int qU = c == 0 ? C_RHOQ : c == 1 ? C_MN : c == 2 ? C_MT1 : c == 3 ? C_MT2 : c == 4 ? C_BT1
                           : c == 5 ? C_BT2 : C_E;
            const Real u0 = SMQ(qU, 0), u1 = SMQ(qU, 1), u2 = SMQ(qU, 2), u3 = SMQ(qU, 3), u4 = SMQ(qU, 4),
                       u5 = SMQ(qU, 5);
            X[6][c] = u1 - u0;
            X[7][c] = u2 - u1;
            X[8][c] = u3 - u2;
            X[9][c] = u4 - u3;
            X[10][c] = u5 - u4;
        }
    }
    // float: the central vector and the pairs (dF_j, du_j) for the packed
    // projection (the same values; only their grouping)
    [[maybe_unused]] float X0f[7];
    [[maybe_unused]] float2 X2f[5][7];
    if constexpr (std::is_same<Real, float>::value) {
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            X0f[c] = X[0][c];
#pragma unroll
            for (int j = 0; j < 5; ++j) X2f[j][c] = make_float2(X[1 + j][c], X[6 + j][c]);
        }
    }
    // interface state: mean of the primitives of cells i and i+1
    const Real r = Real(0.5) * (SMQ(C_RHO, 2) + SMQ(C_RHO, 3));
    const Real vn = Real(0.5) * (SMQ(C_VN, 2) + SMQ(C_VN, 3));
    const Real vt1 = Real(0.5) * (SMQ(C_VT1, 2) + SMQ(C_VT1, 3));
    const Real vt2 = Real(0.5) * (SMQ(C_VT2, 2) + SMQ(C_VT2, 3));
    const Real Bn = Real(0.5) * (SMQ(C_BN, 2) + SMQ(C_BN, 3));
    const Real Bt1 = Real(0.5) * (SMQ(C_BT1, 2) + SMQ(C_BT1, 3));
    const Real Bt2 = Real(0.5) * (SMQ(C_BT2, 2) + SMQ(C_BT2, 3));
    const Real P = Real(0.5) * (SMQ(C_P, 2) + SMQ(C_P, 3));
    // Lax-Friedrichs speeds alpha(m) from the cell eigenvalues
    const Real vL = SMQ(C_VN, 2), vR = SMQ(C_VN, 3);
    const Real cfL = SMQ(C_CF, 2), cfR = SMQ(C_CF, 3);
    const Real caL = SMQ(C_CA, 2), caR = SMQ(C_CA, 3);
    const Real csL = SMQ(C_CSL, 2), csR = SMQ(C_CSL, 3);
    const Real al_fm = m::max_(m::abs_(vL - cfL), m::abs_(vR - cfR));
    const Real al_fp = m::max_(m::abs_(vL + cfL), m::abs_(vR + cfR));
    const Real al_am = m::max_(m::abs_(vL - caL), m::abs_(vR - caR));
    const Real al_ap = m::max_(m::abs_(vL + caL), m::abs_(vR + caR));
    const Real al_sm = m::max_(m::abs_(vL - csL), m::abs_(vR - csR));
    const Real al_sp = m::max_(m::abs_(vL + csL), m::abs_(vR + csR));
    const Real al_e = m::max_(m::abs_(vL), m::abs_(vR));
    // transport fluxes <B_n v_t> of the two cells
    const Real bvt1 = Real(0.5) * (SMQ(C_BN, 2) * SMQ(C_VT1, 2) + SMQ(C_BN, 3) * SMQ(C_VT1, 3));
    const Real bvt2 = Real(0.5) * (SMQ(C_BN, 2) * SMQ(C_VT2, 2) + SMQ(C_BN, 3) * SMQ(C_VT2, 3));
#undef SMQ

    // ---- eigen scalars at the interface state (Appendix A)
    const Real ir = m::rcp_(r);
    const Real ca2 = Bn * Bn * ir;
    const Real btm = Bt1 * Bt1 + Bt2 * Bt2;
    const Real bt2 = btm * ir;
    const Real v2 = vn * vn + vt1 * vt1 + vt2 * vt2;
    // The slow and fast left eigenvectors carry 1/(2 c_s^2): the projection
    // amplifies the rounding of the data by about (v^2 + c_A^2 + b_t^2)/c_s^2.
    // In float, near a pressure floor, that reaches 1e9 and the split fluxes
    // drown in rounding, so the eigenvectors (never the LF speeds) take c_s^2
    // no smaller than cs2_rel times that sum.  L and R stay exact inverses, so
    // the flux stays consistent and conservative; only the basis in which
    // WENO reconstructs changes.  cs2_rel = 0 in double.
    Real cs2 = K.gamma * P * ir;
    if constexpr (float_based<Real>) cs2 = m::max_(cs2, K.cs2_rel * (v2 + ca2 + bt2));
    Real fmc, cms, cf2, csl2;
    speeds_fast<Real>(cs2, ca2, bt2, fmc, cms, cf2);
    const Real sr = m::sqrt_(r);
    const Real isr = sr * ir;
    // c_slow = c_s c_A / c_f (c_slow^2 = c_s^2 c_A^2 / c_f^2), c_A = |B_n| / sqrt(rho)
    const Real cf = m::sqrt_(cf2), cs = m::sqrt_(cs2);
    const Real csl = cf > Real(0) ? cs * (m::abs_(Bn) * isr) * m::rcp_(cf) : Real(0);
    csl2 = csl * csl;
    const Real dfs = fmc + cms;   // c_f^2 - c_slow^2
    Real af, as;
    if (dfs >= K.eps_b2) {
        const Real idf = m::rcp_(dfs);
        af = m::sqrt_(m::max_(cms * idf, Real(0)));
        as = m::sqrt_(m::max_(fmc * idf, Real(0)));
    } else {
        af = Real(1);
        as = Real(1);
    }
    Real b1, b2, bt;   // b = B_t / |B_t|, bt = |B_t|
    if (btm > K.eps_b) {
        const Real ib = m::rsqrt_(btm);
        b1 = Bt1 * ib;
        b2 = Bt2 * ib;
        bt = btm * ib;
    } else {
        b1 = Real(0.70710678118654752440);
        b2 = Real(0.70710678118654752440);
        bt = Real(0);
    }
    const Real sg = (Bn >= K.eps_b) ? Real(1) : Real(-1);
    const Real bv = b1 * vt1 + b2 * vt2;
    const Real Gf = af * cf * vn - as * csl * sg * bv;
    const Real Ga = sg * (b2 * vt1 - b1 * vt2);
    const Real Gs = as * csl * vn + af * cf * sg * bv;
    const Real ics2 = m::rcp_(cs2);
    const Real pre = Real(0.5) * ics2;
    const Real eps = Real(4.0 / 3.0) * K.eps_w;   // 4 eps / 3: see weno_field

    // The sign-free parts of the fast and slow left eigenvectors and the
    // entropy left eigenvector are combinations of two common vectors,
    //   G = (v^2 / 2, -v_n, -v_t1, -v_t2, -B_t1, -B_t2, 1),
    //   H = (0, 0, 0, 0, b_1, b_2, 0):
    //   Lc_fast = pre ((gamma - 1) a_f G + sqrt(rho) c_s a_s H),
    //   Lc_slow = pre ((gamma - 1) a_s G - sqrt(rho) c_s a_f H),
    //   L_entropy = e_0 - (gamma - 1) G / c_s^2   (e_0: the density's unit vector),
    // so each stencil vector is projected on G (its last component, 1, needs
    // no product) and H once.  In double, G's field part -B_t = -|B_t| b is
    // taken as -|B_t| (H.X): G.X = X_E + (v^2/2) X_rho - v.X_m - |B_t| H.X.
    // (Where |B_t|^2 <= eps_B the default b is not B_t / |B_t|; there |B_t| is
    // taken as 0, which leaves out at most |B_t| |X_B| <= 1e-15 |X_B| of G.X.)
    const Real G[7] = {Real(0.5) * v2, -vn, -vt1, -vt2, -Bt1, -Bt2, Real(1)};
    [[maybe_unused]] Real gX[11], hX[11];     // double: G.X, H.X
    [[maybe_unused]] float g0, h0;            // float: the central vector's and
    [[maybe_unused]] float2 g2[5], h2[5];     // the five pairs' projections
    if constexpr (std::is_same<Real, float>::value) {
        // (float: G projected in full -- the H form measured 0.7% slower, its
        // longer-lived projections spilling more)
        constexpr int cc[7] = {0, 1, 2, 3, 4, 5, 6};
        constexpr int ch[2] = {4, 5};
        const float Hc[2] = {b1, b2};
        project_f<7>(X0f, X2f, cc, G, g0, g2);   // (the compiler drops the factor 1)
        project_f<2>(X0f, X2f, ch, Hc, h0, h2);
    } else {
#pragma unroll
        for (int x = 0; x < 11; ++x) {
            const Real hx = b1 * X[x][4] + b2 * X[x][5];
            Real gx = X[x][6] + G[0] * X[x][0];
#pragma unroll
            for (int c = 1; c < 4; ++c) gx += G[c] * X[x][c];
            gX[x] = gx - bt * hx;
            hX[x] = hx;
        }
    }
    // The WENO fluxes (Fu for the left eigenvector Lc + Ls, Fl for Lc - Ls)
    // of one magnetosonic pair: Lc = cg G + ch H, Ls non-zero in rows 0..3.
    auto magnetosonic = [&](Real cg, Real ch, const Real (&Ls)[4], Real alu, Real all, Real &Fu, Real &Fl) {
        Real Pu[11], Pl[11];
        if constexpr (std::is_same<Real, float>::value) {
            constexpr int cs4[4] = {0, 1, 2, 3};
            const float pc0 = cg * g0 + ch * h0;
            float2 pc2[5];
#pragma unroll
            for (int j = 0; j < 5; ++j) pc2[j] = __ffma2_rn(bcast2(cg), g2[j], __fmul2_rn(bcast2(ch), h2[j]));
            float ps0;
            float2 ps2[5];
            project_f<4>(X0f, X2f, cs4, Ls, ps0, ps2);
            split_pair_f(pc0, pc2, ps0, ps2, Pu, Pl);
        } else {
#pragma unroll
            for (int x = 0; x < 11; ++x) {
                const Real pc = cg * gX[x] + ch * hX[x];
                Real ps = Ls[0] * X[x][0];
#pragma unroll
                for (int c = 1; c < 4; ++c) ps += Ls[c] * X[x][c];
                Pu[x] = pc + ps;
                Pl[x] = pc - ps;
            }
        }
        Fu = weno_field<Real, VAR, DWW>(Pu, alu, eps);
        Fl = weno_field<Real, VAR, DWW>(Pl, all, eps);
    };

    // ---- fast pair: m = 1 (v - c_f, upper sign) and m = 7 (v + c_f)
    Real sf, df;
    {
        const Real Ls[4] = {pre * Gf, -pre * af * cf, pre * csl * as * b1 * sg, pre * csl * as * b2 * sg};
        Real Fu, Fl;
        magnetosonic(pre * (K.gm1 * af), pre * (sr * cs * as), Ls, al_fm, al_fp, Fu, Fl);
        sf = Fu + Fl;
        df = Fu - Fl;
    }
    // ---- slow pair: m = 3 (v - c_slow, upper sign) and m = 5 (v + c_slow)
    Real ss, ds;
    {
        const Real Ls[4] = {pre * Gs, -pre * as * csl, -pre * cf * af * b1 * sg, -pre * cf * af * b2 * sg};
        Real Fu, Fl;
        magnetosonic(pre * (K.gm1 * as), -(pre * (sr * cs * af)), Ls, al_sm, al_sp, Fu, Fl);
        ss = Fu + Fl;
        ds = Fu - Fl;
    }
    // ---- Alfven pair: m = 2 (v - c_A, upper sign) and m = 6 (v + c_A)
    //   L = (Ga/2, 0, -b2 sg/2, b1 sg/2, -+ sr b2/2, +- sr b1/2, 0)
    //   R = (0, 0, -b2 sg, b1 sg, -+ b2/sr, +- b1/sr, -Ga)
    Real sa, da;
    {
        const Real l0 = Real(0.5) * Ga, l2 = Real(-0.5) * b2 * sg, l3 = Real(0.5) * b1 * sg;
        const Real l4 = Real(-0.5) * sr * b2, l5 = Real(0.5) * sr * b1;
        Real Pu[11], Pl[11];
        if constexpr (std::is_same<Real, float>::value) {
            constexpr int cc[3] = {0, 2, 3};
            constexpr int cs[2] = {4, 5};
            const float Lc[3] = {l0, l2, l3}, Ls[2] = {l4, l5};
            float pc0, ps0;
            float2 pc2[5], ps2[5];
            project_f<3>(X0f, X2f, cc, Lc, pc0, pc2);
            project_f<2>(X0f, X2f, cs, Ls, ps0, ps2);
            split_pair_f(pc0, pc2, ps0, ps2, Pu, Pl);
        } else {
#pragma unroll
            for (int x = 0; x < 11; ++x) {
                const Real pc = l0 * X[x][0] + l2 * X[x][2] + l3 * X[x][3];
                const Real ps = l4 * X[x][4] + l5 * X[x][5];
                Pu[x] = pc + ps;
                Pl[x] = pc - ps;
            }
        }
        const Real Fu = weno_field<Real, VAR, DWW>(Pu, al_am, eps);
        const Real Fl = weno_field<Real, VAR, DWW>(Pl, al_ap, eps);
        sa = Fu + Fl;
        da = Fu - Fl;
    }
    // ---- entropy field: m = 4 (v), L = e_0 - (gamma - 1) G / c_s^2
    Real Fe;
    {
        const Real tau = K.gm1 * ics2;
        Real Pe[11];
        if constexpr (std::is_same<Real, float>::value) {
            float2 pe2[5];
#pragma unroll
            for (int j = 0; j < 5; ++j) pe2[j] = __ffma2_rn(bcast2(-tau), g2[j], X2f[j][0]);
            unpack11(__fmaf_rn(-tau, g0, X0f[0]), pe2, Pe);
        } else {
#pragma unroll
            for (int x = 0; x < 11; ++x) Pe[x] = X[x][0] - tau * gX[x];
        }
        Fe = weno_field<Real, VAR, DWW>(Pe, al_e, eps);
    }
    // ---- back-projection: F = sum over fields of (WENO flux) x (right
    // eigenvector).  The right eigenvectors of the fast pair (Rc +- Rs),
    //   Rc = (a_f, a_f v, c_s a_s b / sqrt(rho), a_f (v^2/2 + c_f^2 - g2 c_s^2)),
    //   Rs = rows (1, 2, 3, 6): (-a_f c_f, c_slow a_s b sg, -Gf),
    // of the slow pair (a_f, c_f -> a_s, c_slow and a_s, c_slow -> -a_f, c_f
    // in Rc's field rows and Rs) and of the entropy field (1, v, 0, v^2 / 2)
    // share R1 = (1, v, 0, 0, v^2/2 - g2 c_s^2) and (0, 0, 0, 0, b_1, b_2, 0),
    // so the sums (Fu + Fl) and differences (Fu - Fl) of the fields combine
    // into a few scalars first.
    {
        const Real S1 = af * sf + as * ss + Fe;
        const Real S2 = (cs * isr) * (as * sf - af * ss);
        const Real T1 = -(af * cf * df + as * csl * ds);
        const Real T2 = sg * (csl * as * df - cf * af * ds);
        const Real w = Real(0.5) * v2 - K.g2 * cs2;
        Ff[0] = S1;
        Ff[1] = S1 * vn + T1;
        Ff[2] = S1 * vt1 + T2 * b1 - sa * (b2 * sg);
        Ff[3] = S1 * vt2 + T2 * b2 + sa * (b1 * sg);
        Ff[4] = S2 * b1 - da * (b2 * isr);
        Ff[5] = S2 * b2 + da * (b1 * isr);
        Ff[6] = S1 * w + af * cf2 * sf + as * csl2 * ss + K.g2 * cs2 * Fe - (Gf * df + Gs * ds) - sa * Ga;
    }
    s1 = Ff[4] + bvt1;
    s2 = Ff[5] + bvt2;
}

}  // namespace w5ct
