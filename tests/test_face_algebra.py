"""The face arithmetic of the sweep kernels, restated and checked against the
oracle's Appendix A eigensystem and phi_N (Sec. 2.2) on the CPU.

The kernels do not form the seven left and right eigenvectors row by row.
They use combinations of them that are exact in exact arithmetic:

* the sign-free parts of the fast and slow left eigenvectors and the entropy
  left eigenvector are combinations of G = (v^2/2, -v, -B_t, 1) and
  H = (0, 0, 0, 0, b_1, b_2, 0);
* the frame flux sum_m F_m R_m is assembled from six scalars of the field
  fluxes;
* phi_N = [a_0 t1 + (a_2/2 - D/4) t2] / (3 D) with the WENO weights scaled
  by (s_0 s_1 s_2)^2 (FP64) or normalised (float), t1, t2 the second
  differences, eps inside the smoothness indicators.

These tests restate those formulas in NumPy and compare them with the
oracle, so that a slip in the restructured algebra (a dropped term, a wrong
sign, a swapped pair member) fails here, independently of the GPU.
"""
import numpy as np
import pytest

import oracle as ora

GAMMA = 5.0 / 3.0


def random_states(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        rho = rng.uniform(0.2, 3.0)
        v = rng.normal(0.0, 1.0, 3)
        Bn = rng.choice([-1.0, 1.0]) * rng.uniform(0.1, 2.0)
        Bt = rng.normal(0.0, 1.0, 2)
        P = rng.uniform(0.05, 3.0)
        out.append(np.array([rho, v[0], v[1], v[2], Bn, Bt[0], Bt[1], P]))
    return out


def kernel_eigen(w, gamma=GAMMA):
    """The interface scalars of the sweep kernels (face function) at w."""
    r, vn, vt1, vt2, Bn, Bt1, Bt2, P = w
    gm1, g2 = gamma - 1.0, (gamma - 2.0) / (gamma - 1.0)
    ir = 1.0 / r
    ca2, btm = Bn * Bn * ir, Bt1 * Bt1 + Bt2 * Bt2
    bt2, v2 = btm * ir, vn * vn + vt1 * vt1 + vt2 * vt2
    cs2 = gamma * P * ir
    dd = (cs2 - ca2) ** 2 + bt2 * (bt2 + 2 * ca2 + 2 * cs2)
    sd, aa = np.sqrt(dd), ca2 + bt2 - cs2
    if aa >= 0:
        fmc = 0.5 * (aa + sd)
        cms = cs2 * bt2 / fmc
    else:
        cms = 0.5 * (sd - aa)
        fmc = cs2 * bt2 / cms
    cf2 = cs2 + fmc
    sr = np.sqrt(r)
    isr = sr * ir
    cf, cs = np.sqrt(cf2), np.sqrt(cs2)
    csl = cs * (abs(Bn) * isr) / cf          # c_slow = c_s c_A / c_f
    csl2 = csl * csl
    dfs = fmc + cms
    af, as_ = np.sqrt(cms / dfs), np.sqrt(fmc / dfs)
    b1, b2 = Bt1 / np.sqrt(btm), Bt2 / np.sqrt(btm)
    sg = 1.0 if Bn >= 0 else -1.0
    bv = b1 * vt1 + b2 * vt2
    return dict(vn=vn, vt1=vt1, vt2=vt2, v2=v2, cf=cf, cs=cs, csl=csl, cf2=cf2, csl2=csl2, cs2=cs2, af=af,
                as_=as_, b1=b1, b2=b2, sg=sg, sr=sr, isr=isr, gm1=gm1, g2=g2, pre=0.5 / cs2,
                Gf=af * cf * vn - as_ * csl * sg * bv, Gs=as_ * csl * vn + af * cf * sg * bv,
                Ga=sg * (b2 * vt1 - b1 * vt2), Bt1=Bt1, Bt2=Bt2)


def test_kernel_slow_speed_equals_the_oracle_wave_speeds():
    for w in random_states(200, 11):
        e = kernel_eigen(w)
        cs, ca, csl, cf = ora.wave_speeds(w, GAMMA)
        np.testing.assert_allclose([e["cs"], e["csl"], e["cf"]], [cs, csl, cf], rtol=1e-13)


def test_left_eigenvectors_from_the_shared_vectors():
    """Lc_fast = pre((gamma-1) a_f G + sqrt(rho) c_s a_s H), Lc_slow = pre((gamma-1)
    a_s G - sqrt(rho) c_s a_f H), L_entropy = e_0 - (gamma-1) G / c_s^2, and the
    sign-dependent parts Ls and the Alfven pair, against the oracle's rows
    (m = 1..7: v - c_f, v - c_A, v - c_slow, v, v + c_slow, v + c_A, v + c_f)."""
    for w in random_states(200, 12):
        L, R, lam = ora.eigensystem(w, GAMMA)
        e = kernel_eigen(w)
        G = np.array([0.5 * e["v2"], -e["vn"], -e["vt1"], -e["vt2"], -e["Bt1"], -e["Bt2"], 1.0])
        H = np.array([0, 0, 0, 0, e["b1"], e["b2"], 0.0])
        pre, gm1 = e["pre"], e["gm1"]
        scale = np.abs(L).max()
        # fast pair: rows 0 (upper) and 6 (lower)
        Lc = pre * (gm1 * e["af"] * G + e["sr"] * e["cs"] * e["as_"] * H)
        Ls = pre * np.array([e["Gf"], -e["af"] * e["cf"], e["csl"] * e["as_"] * e["b1"] * e["sg"],
                             e["csl"] * e["as_"] * e["b2"] * e["sg"], 0, 0, 0])
        np.testing.assert_allclose(Lc + Ls, L[0], atol=1e-12 * scale)
        np.testing.assert_allclose(Lc - Ls, L[6], atol=1e-12 * scale)
        # slow pair: rows 2 (upper) and 4 (lower)
        Lc = pre * (gm1 * e["as_"] * G - e["sr"] * e["cs"] * e["af"] * H)
        Ls = pre * np.array([e["Gs"], -e["as_"] * e["csl"], -e["cf"] * e["af"] * e["b1"] * e["sg"],
                             -e["cf"] * e["af"] * e["b2"] * e["sg"], 0, 0, 0])
        np.testing.assert_allclose(Lc + Ls, L[2], atol=1e-12 * scale)
        np.testing.assert_allclose(Lc - Ls, L[4], atol=1e-12 * scale)
        # Alfven pair: rows 1 (upper) and 5 (lower)
        Lc = np.array([0.5 * e["Ga"], 0, -0.5 * e["b2"] * e["sg"], 0.5 * e["b1"] * e["sg"], 0, 0, 0])
        Ls = np.array([0, 0, 0, 0, -0.5 * e["sr"] * e["b2"], 0.5 * e["sr"] * e["b1"], 0])
        np.testing.assert_allclose(Lc + Ls, L[1], atol=1e-12 * scale)
        np.testing.assert_allclose(Lc - Ls, L[5], atol=1e-12 * scale)
        # entropy: row 3
        e0 = np.array([1.0, 0, 0, 0, 0, 0, 0])
        np.testing.assert_allclose(e0 - gm1 * G / e["cs2"], L[3], atol=1e-12 * scale)


def kernel_back_projection(Fm, e):
    """The sweep kernels' frame flux from the seven field fluxes
    (Fm[m], rows as in the oracle)."""
    sf, df = Fm[0] + Fm[6], Fm[0] - Fm[6]
    ss, ds = Fm[2] + Fm[4], Fm[2] - Fm[4]
    sa, da = Fm[1] + Fm[5], Fm[1] - Fm[5]
    Fe = Fm[3]
    af, as_, cf, csl, cs, isr = e["af"], e["as_"], e["cf"], e["csl"], e["cs"], e["isr"]
    b1, b2, sg = e["b1"], e["b2"], e["sg"]
    S1 = af * sf + as_ * ss + Fe
    S2 = (cs * isr) * (as_ * sf - af * ss)
    T1 = -(af * cf * df + as_ * csl * ds)
    T2 = sg * (csl * as_ * df - cf * af * ds)
    w = 0.5 * e["v2"] - e["g2"] * e["cs2"]
    return np.array([
        S1,
        S1 * e["vn"] + T1,
        S1 * e["vt1"] + T2 * b1 - sa * (b2 * sg),
        S1 * e["vt2"] + T2 * b2 + sa * (b1 * sg),
        S2 * b1 - da * (b2 * isr),
        S2 * b2 + da * (b1 * isr),
        S1 * w + af * e["cf2"] * sf + as_ * e["csl2"] * ss + e["g2"] * e["cs2"] * Fe - (e["Gf"] * df + e["Gs"] * ds)
        - sa * e["Ga"],
    ])


def test_back_projection_equals_the_sum_over_right_eigenvectors():
    rng = np.random.default_rng(13)
    for w in random_states(200, 14):
        L, R, lam = ora.eigensystem(w, GAMMA)
        e = kernel_eigen(w)
        Fm = rng.normal(0.0, 1.0, 7)
        want = Fm @ R
        np.testing.assert_allclose(kernel_back_projection(Fm, e), want, atol=1e-12 * np.abs(R).max())


def kernel_phi_fp64(a, b, c, d, eps, Z):
    """phi_N as the FP64 kernels evaluate it (weights times (s0 s1 s2)^2)."""
    k, e3 = 13.0 / 3.0, eps / 3.0
    x0, y0, z0 = a - b, b - c, c - d
    s0 = k * x0 * x0 + ((a - 3 * b) ** 2 + e3)
    s1 = k * y0 * y0 + ((b + c) ** 2 + e3)
    s2 = k * z0 * z0 + ((3 * c - d) ** 2 + e3)
    if Z:
        tt = (s0 - s2) ** 2
        e0, e1, e2 = s0 * s0, s1 * s1, s2 * s2
        E = e0 * e1 * e2
        W0, V1, V2 = tt * e1 * e2 + E, tt * e0 * e2 + E, tt * e0 * e1 + E
    else:
        W0, V1, V2 = (s1 * s2) ** 2, (s0 * s2) ** 2, (s0 * s1) ** 2
    D = W0 + 6 * V1 + 3 * V2
    N = W0 * (x0 - y0) + (1.5 * V2 - 0.25 * D) * (y0 - z0)
    return N / (3 * D)


def kernel_phi_float(a, b, c, d, eps, Z):
    """phi_N as the float kernels evaluate it (normalised weights), in double."""
    k, e3 = 13.0 / 3.0, eps / 3.0
    x0, y0, z0 = a - b, b - c, c - d
    s = [k * x0 * x0 + ((a - 3 * b) ** 2 + e3), k * y0 * y0 + ((b + c) ** 2 + e3),
         k * z0 * z0 + ((3 * c - d) ** 2 + e3)]
    if Z:
        tau = abs(s[0] - s[2])
        e = [1 + min(tau / sk, 1e18) ** 2 for sk in s]
    else:
        e = [1 / (sk * sk) for sk in s]
    inv = 1 / (e[0] + 6 * e[1] + 3 * e[2])
    return ((e[0] * inv) * (x0 - y0) + (e[2] * 1.5 * inv - 0.25) * (y0 - z0)) / 3


@pytest.mark.parametrize("Z", [0, 1])
def test_phi_n_forms_equal_the_oracle(Z):
    rng = np.random.default_rng(15 + Z)
    cfg = ora.make_config(weno_variant=Z)
    eps = cfg.eps_z if Z else cfg.eps_js
    worst64 = worst32 = 0.0
    for _ in range(2000):
        v = rng.normal(0.0, 1.0, 4) * rng.choice([1e-3, 1.0, 1e3])
        want = ora.phi_n(*v, cfg)
        scale = np.abs(v).max()
        worst64 = max(worst64, abs(kernel_phi_fp64(*v, eps, Z) - want) / scale)
        worst32 = max(worst32, abs(kernel_phi_float(*v, eps, Z) - want) / scale)
    assert worst64 < 1e-13, worst64
    assert worst32 < 1e-13, worst32


def kernel_phi_dw_form(a, b, c, d, eps, Z):
    """phi_N as the double-word FP64 sweeps evaluate it (weno_field with the
    double-word flag), in float64: the weights relative to the smallest
    indicator s_m, rho_k = s_m / s_k, JS e_k = rho_k^2, WENO-Z e_k =
    1 + (R rho_k)^2 with R = tau / s_m, or (R rho_k)^2 scaled by 1/R^2 where
    R > 1e18.  An epsilon below float's normal range is 0 there."""
    e3 = eps / 3.0
    if e3 < 2.0 ** -126:
        e3 = 0.0
    k = 13.0 / 3.0
    x0, y0, z0 = a - b, b - c, c - d
    x1, y1, z1 = x0 - 2 * b, b + c, z0 + 2 * c
    s = [k * x0 * x0 + x1 * x1 + e3, k * y0 * y0 + y1 * y1 + e3, k * z0 * z0 + z1 * z1 + e3]
    s = [0.0 if sk < 2.0 ** -126 else sk for sk in s]     # below float's normal range: flat
    sm = min(s)
    rho = [1.0 if sk == sm else sm / sk for sk in s]
    e = [r * r for r in rho]
    if Z:
        tau = abs(s[0] - s[2])
        R = 0.0 if tau == 0.0 else (tau / sm if sm > 0 else np.inf)
        if R <= 1e18:
            e = [1.0 + R * R * ek for ek in e]
    D = e[0] + 6 * e[1] + 3 * e[2]
    return ((e[0] / D) * (x0 - y0) + (1.5 * e[2] / D - 0.25) * (y0 - z0)) / 3


@pytest.mark.parametrize("Z", [0, 1])
def test_phi_n_double_word_form_equals_the_oracle(Z):
    """The ratio-to-the-smallest-indicator weights, on random stencils of
    every scale and on stencils with flat parts (indicators at epsilon, or
    0 where epsilon is below float's range), against the oracle's phi_N."""
    rng = np.random.default_rng(31 + Z)
    cfg = ora.make_config(weno_variant=Z)
    eps = cfg.eps_z if Z else cfg.eps_js
    cases = [rng.normal(0.0, 1.0, 4) * rng.choice([1e-6, 1e-3, 1.0, 1e3]) for _ in range(2000)]
    cases += [np.array(v, dtype=float) for v in
              ([1.0, 0, 0, 0], [0, 0, 0, 1.0], [0, 1.0, 0, 0], [0, 0, 1.0, 0], [1.0, 1.0, 0, 0], [2.0, 0, 0, -1.0],
               [0, 0, 0, 0], [1e-3, 2e-3, 0, 0], [3.0, 1.0, 1.0, 3.0], [1.0, 1.0, 1.0, 1.0], [1e-20, 0, 0, 5.0],
               [1e-21, -2e-21, 3e-21, 1.0], [1.0, 1e-21, -1e-21, 2e-21])]
    worst = 0.0
    for v in cases:
        want = ora.phi_n(*v, cfg)
        got = kernel_phi_dw_form(*v, eps, Z)
        worst = max(worst, abs(got - want) / max(np.abs(v).max(), 1e-300))
    assert worst < 1e-13, worst
    # stencils whose differences are all below 1e-19 count as flat; there the
    # double weights are set by rounding noise, and phi_N agrees in absolute
    # terms (far below any flux of an O(1) state)
    for v in ([2e-22, 1e-21, -1e-21, 3e-22], [-3e-21, 2e-21, 5e-22, -1e-21]):
        v = np.array(v)
        assert abs(kernel_phi_dw_form(*v, eps, Z) - ora.phi_n(*v, cfg)) < 1e-20
