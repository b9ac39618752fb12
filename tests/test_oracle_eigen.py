"""Pins of the oracle's eigen-algebra (Appendix A) and flux (Eq. fluxes).

* the right eigenvectors and eigenvalues printed for the linear-wave
  background (Sec. 4.1) -- golden fixture;
* L R = I at generic and degenerate states;
* A R = R Lambda and L A = Lambda L with A the complex-step Jacobian of the
  conservative flux, and the finite-difference Jacobian of the oracle's own
  flux having the oracle's eigenvalues.
"""
import os

import numpy as np
import pytest

G = 5.0 / 3.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "linear_wave_eigenvectors.txt")


def _num(tok):
    """Parse a printed entry: integers, fractions, 'r2' = sqrt2, 'r5' = sqrt5,
    'gamma' (e.g. '-4r2', '1/(6r5)', '1/(gamma-1)')."""
    t = tok.replace("gamma", "(%r)" % float(G))
    for name, val in (("r2", float(np.sqrt(2.0))), ("r5", float(np.sqrt(5.0)))):
        out = ""
        i = 0
        while i < len(t):
            if t.startswith(name, i):
                prev = out[-1] if out else ""
                out += ("*" if prev.isdigit() or prev == ")" else "") + "(%r)" % val
                i += len(name)
            else:
                out += t[i]
                i += 1
        t = out
    return float(eval(t, {"__builtins__": {}}))


def golden_vectors():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        out[parts[0]] = _num(parts[1]) * np.array([_num(t) for t in parts[2:]])
    return out


def drop_bx(v8):
    return np.delete(v8, 4)


def test_worked_example_eigenvalues_and_vectors(ora):
    gv = golden_vectors()
    w = np.array([1.0, 0.0, 0.0, 0.0, 1.0, np.sqrt(2.0), 0.5, 1.0 / G])
    L, R, lam = ora.eigensystem(w, G)
    np.testing.assert_allclose(lam, [-2, -1, -0.5, 0, 0.5, 1, 2], atol=1e-15)
    # m = 7 (v + c_f) is the printed fast vector, m = 5 (v + c_slow) the slow one
    np.testing.assert_allclose(R[6], drop_bx(gv["fast"]), atol=1e-15, rtol=0)
    np.testing.assert_allclose(R[4], drop_bx(gv["slow"]), atol=1e-15, rtol=0)
    # m = 6 (v + c_A) is the printed Alfven vector up to the factor -2 sqrt5
    np.testing.assert_allclose(R[5], -2.0 * np.sqrt(5.0) * drop_bx(gv["alfven"]), atol=1e-15, rtol=0)
    # none of the printed vectors has a B_x component
    for k in ("fast", "slow", "alfven"):
        assert gv[k][4] == 0.0


def test_worked_example_hydro_vectors(ora):
    gv = golden_vectors()
    # entropy mode at v_x = 1, B = 0 (this pins the energy row v^2/2 of R_entropy)
    w = np.array([1.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0 / G])
    L, R, lam = ora.eigensystem(w, G)
    np.testing.assert_allclose(R[3], drop_bx(gv["entropy"]), atol=1e-15)
    # sound wave at v = 0, B = 0 is the fast mode m = 7 (c_f = c_s = 1)
    w = np.array([1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0 / G])
    L, R, lam = ora.eigensystem(w, G)
    np.testing.assert_allclose(lam[6], 1.0, atol=1e-15)
    np.testing.assert_allclose(R[6], drop_bx(gv["sound"]), atol=1e-15)


def random_states(rng, n):
    out = []
    for _ in range(n):
        rho = rng.uniform(0.2, 3.0)
        v = rng.normal(0, 1.0, 3)
        B = rng.normal(0, 1.5, 3)
        P = rng.uniform(0.05, 3.0)
        out.append(np.array([rho, *v, *B, P]))
    return out


def degenerate_states():
    s = []
    # B_n = 0 (sgn = -1 branch), B_t != 0
    s.append(np.array([1.3, 0.2, -0.4, 0.1, 0.0, 0.7, -0.3, 0.9]))
    # B_t = 0, c_A > c_s and c_A < c_s
    s.append(np.array([1.0, 0.3, 0.1, -0.2, 2.0, 0.0, 0.0, 0.6]))
    s.append(np.array([1.0, 0.3, 0.1, -0.2, 0.2, 0.0, 0.0, 0.6]))
    # B = 0 (hydro)
    s.append(np.array([0.7, -0.5, 0.2, 0.9, 0.0, 0.0, 0.0, 1.1]))
    # negative B_n
    s.append(np.array([1.1, 0.0, 0.5, 0.5, -0.8, 0.4, 0.9, 0.4]))
    # tiny B_t (near the beta default threshold)
    s.append(np.array([1.0, 0.1, 0.0, 0.0, 1.5, 1e-9, -2e-9, 1.0]))
    return s


def lr_error(ora, w):
    L, R, lam = ora.eigensystem(w, G)
    return np.abs(L @ R.T - np.eye(7)).max()


def test_left_right_inverse(ora):
    rng = np.random.default_rng(7)
    for w in random_states(rng, 200) + degenerate_states():
        assert lr_error(ora, w) < 1e-12, w


def test_near_triple_point(ora):
    # c_A = c_s and |B_t| -> 0: the eigenvector basis stays well defined
    rho, P = 1.0, 0.6
    Bn = np.sqrt(G * P)          # c_A = c_s
    for bt in (1e-3, 1e-6):
        w = np.array([rho, 0.1, 0.2, -0.1, Bn, bt, 0.5 * bt, P])
        assert lr_error(ora, w) < 1e-7


def test_exact_triple_point_takes_fallback(ora):
    # c_f = c_slow exactly: Appendix A sets alpha_f = alpha_s = 1
    rho, P = 1.0, 0.6
    Bn = 1.0
    P = Bn * Bn / G              # c_s^2 = gamma P / rho = B_n^2 / rho = c_A^2
    w = np.array([rho, 0.0, 0.0, 0.0, Bn, 0.0, 0.0, P])
    L, R, lam = ora.eigensystem(w, G)
    assert R[0][0] == 1.0 and R[2][0] == 1.0     # alpha_f = alpha_s = 1
    assert np.all(np.isfinite(L)) and np.all(np.isfinite(R))


# ---------------------------------------------------------------- Jacobian


def conservative_flux(u, Bn, gamma=G):
    """Ideal-MHD flux along n of u = (rho, m_n, m_t1, m_t2, B_t1, B_t2, E),
    written in vector form (complex-safe)."""
    rho = u[0]
    m = np.array([u[1], u[2], u[3]])
    B = np.array([Bn + 0 * u[0], u[4], u[5]])
    E = u[6]
    v = m / rho
    P = (gamma - 1.0) * (E - 0.5 * np.sum(m * v) - 0.5 * np.sum(B * B))
    Pt = P + 0.5 * np.sum(B * B)
    n = np.array([1.0, 0.0, 0.0])
    mom = m * v[0] + Pt * n - B * B[0]
    induc = B * v[0] - v * B[0]
    en = (E + Pt) * v[0] - B[0] * np.sum(v * B)
    return np.array([m[0], mom[0], mom[1], mom[2], induc[1], induc[2], en])


def prim_to_u(w, gamma=G):
    rho, vn, v1, v2, Bn, B1, B2, P = w
    E = P / (gamma - 1) + 0.5 * rho * (vn * vn + v1 * v1 + v2 * v2) + 0.5 * (Bn * Bn + B1 * B1 + B2 * B2)
    return np.array([rho, rho * vn, rho * v1, rho * v2, B1, B2, E])


def u_to_prim(u, Bn, gamma=G):
    rho = u[0]
    v = u[1:4] / rho
    B2 = Bn * Bn + u[4] ** 2 + u[5] ** 2
    P = (gamma - 1) * (u[6] - 0.5 * rho * np.sum(v * v) - 0.5 * B2)
    return np.array([rho, v[0], v[1], v[2], Bn, u[4], u[5], P])


def complex_step_jacobian(u, Bn, h=1e-30):
    A = np.zeros((7, 7))
    for j in range(7):
        du = np.zeros(7, dtype=complex)
        du[j] = 1j * h
        A[:, j] = np.imag(conservative_flux(u.astype(complex) + du, Bn)) / h
    return A


def test_jacobian_eigenpairs(ora):
    rng = np.random.default_rng(11)
    for w in random_states(rng, 60) + degenerate_states()[:5]:
        L, R, lam = ora.eigensystem(w, G)
        A = complex_step_jacobian(prim_to_u(w), w[4])
        scale = np.abs(A).max() * max(1.0, np.abs(R).max()) * max(1.0, np.abs(L).max())
        for m in range(7):
            assert np.abs(A @ R[m] - lam[m] * R[m]).max() < 1e-12 * scale, (w, m)
            assert np.abs(L[m] @ A - lam[m] * L[m]).max() < 1e-12 * scale, (w, m)


def test_oracle_flux_jacobian_spectrum(ora):
    """The finite-difference Jacobian of the oracle's own flux has the
    oracle's eigenvalues and eigenvectors (pins Eq. fluxes and the speeds)."""
    rng = np.random.default_rng(5)
    for w in random_states(rng, 30):
        u = prim_to_u(w)
        Bn = w[4]

        def F(uu):
            ww = u_to_prim(uu, Bn)
            return ora.frame_flux(ww, uu[6])

        A = np.zeros((7, 7))
        for j in range(7):
            h = 1e-6 * max(1.0, abs(u[j]))
            e = np.zeros(7)
            e[j] = h
            A[:, j] = (F(u + e) - F(u - e)) / (2 * h)
        # flux itself equals the vector-form flux
        np.testing.assert_allclose(F(u), conservative_flux(u, Bn), rtol=1e-13, atol=1e-13)
        L, R, lam = ora.eigensystem(w, G)
        ev = np.sort(np.linalg.eigvals(A).real)
        np.testing.assert_allclose(ev, lam, rtol=1e-6, atol=1e-6)
        for m in range(7):
            np.testing.assert_allclose(A @ R[m], lam[m] * R[m], atol=1e-6 * (1 + np.abs(R[m]).max() * np.abs(A).max()))


def test_wave_speed_orderings(ora):
    rng = np.random.default_rng(3)
    for w in random_states(rng, 200):
        cs, ca, cslow, cf = ora.wave_speeds(w, G)
        assert cslow <= ca * (1 + 1e-14) + 1e-300 and ca <= cf * (1 + 1e-14)
        assert cslow <= cs * (1 + 1e-14) and cs <= cf * (1 + 1e-14)
        B2 = w[4] ** 2 + w[5] ** 2 + w[6] ** 2
        np.testing.assert_allclose(cf ** 2 + cslow ** 2, cs ** 2 + B2 / w[0], rtol=1e-13)


def test_wave_speeds_high_precision(ora):
    """c_f, c_slow against the paper's root formula evaluated to 50 digits
    (Eqs. slow, fast with the 1/2 on the whole bracket)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(4)
    states = random_states(rng, 100) + degenerate_states()
    # strongly separated speeds: c_slow << c_s
    states.append(np.array([1.0, 0.0, 0.0, 0.0, 1e-3, 2.0, 0.0, 1.0]))
    states.append(np.array([1.0, 0.0, 0.0, 0.0, 2.0, 1e-4, 0.0, 0.01]))
    for w in states:
        cs, ca, cslow, cf = ora.wave_speeds(w, G)
        rho, P = mp.mpf(w[0]), mp.mpf(w[7])
        Bn, B1, B2 = (mp.mpf(x) for x in w[4:7])
        cs2 = mp.mpf(G) * P / rho
        Bsq = (Bn * Bn + B1 * B1 + B2 * B2) / rho
        disc = mp.sqrt((Bsq + cs2) ** 2 - 4 * cs2 * Bn * Bn / rho)
        cf_ref = mp.sqrt((cs2 + Bsq + disc) / 2)
        csl_ref = mp.sqrt(max((cs2 + Bsq - disc) / 2, mp.mpf(0)))
        assert abs(cf - float(cf_ref)) <= 4e-16 * float(cf_ref)
        assert abs(cslow - float(csl_ref)) <= 4e-15 * float(csl_ref) + 1e-300
        assert abs(ca - float(abs(Bn) / mp.sqrt(rho))) <= 4e-16 * ca + 1e-300
