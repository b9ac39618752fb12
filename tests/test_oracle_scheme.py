"""Scheme-level pins of the oracle (Secs. 2.1, 2.3, 3.1, 4.1):

* the RK4 stage machinery reproduces the RK4 amplification polynomial;
* a uniform state is preserved (free-stream);
* mass, momentum, energy and the face-field totals are conserved;
* the discrete divergence of b stays at round-off;
* a 3-D state that varies along one axis only evolves exactly like the
  1-D program (no CT), for each of the three axes;
* a cyclic relabelling of the axes commutes with the step;
* linear waves converge at the orders the paper reports.
"""
import numpy as np
import pytest

import oracle as O
from paper_1812_04278_gb300 import inputs as I

G = 5.0 / 3.0


def state_scale(cons, bface):
    return max(np.abs(cons).max(), np.abs(bface).max())


# ------------------------------------------------------------------ RK4


def test_rk4_amplification_polynomial():
    M = np.array([[-0.7, 2.3], [-1.9, 0.4]])   # complex-conjugate eigenvalues
    dt = 0.37
    o = O.Oracle((2, 2, 2), 0.5)
    rng = np.random.default_rng(0)
    cons = rng.normal(size=(5, 2, 2, 2))
    bface = rng.normal(size=(3, 2, 2, 2))
    o.set_state(cons, bface)
    o.step_linear(dt, M)
    c1, b1, _ = o.get_state()
    Z = dt * M
    P = np.eye(2) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
    q0 = np.stack([cons[0].ravel(), cons[1].ravel()])
    np.testing.assert_allclose(np.stack([c1[0].ravel(), c1[1].ravel()]), P @ q0, rtol=0, atol=1e-14)
    np.testing.assert_allclose(c1[2:], cons[2:], rtol=0, atol=1e-15)
    np.testing.assert_array_equal(b1, bface)      # Omega = 0 leaves b untouched


# ------------------------------------------------------------------ invariants


def test_freestream():
    shape = (8, 6, 5)
    cons, bface = I.uniform_state(shape, rho=1.2, v=(0.3, -0.2, 0.5), B=(0.7, -0.4, 0.9), P=0.8)
    o = O.Oracle(shape, (0.1, 0.2, 0.15))
    o.set_state(cons, bface)
    for _ in range(10):
        o.step(o.cfl_dt())
    c1, b1, _ = o.get_state()
    np.testing.assert_array_equal(b1, bface)
    for f in range(5):
        np.testing.assert_allclose(c1[f], cons[f], rtol=4e-15, atol=4e-15 * np.abs(cons[f]).max())


@pytest.fixture(scope="module")
def smooth_run():
    shape = (12, 10, 8)
    cons, bface = I.random_smooth_state(shape, seed=42)
    o = O.Oracle(shape, (1 / 12, 1 / 10, 1 / 8))
    o.set_state(cons, bface)
    tot0 = o.conserved_totals()
    abs0 = np.array([np.abs(cons[f]).sum() for f in range(5)] + [np.abs(bface[f]).sum() for f in range(3)])
    abs0 *= (1 / 12) * (1 / 10) * (1 / 8)
    div0 = o.div_b_norm()
    tots = []
    divs = []
    for _ in range(3):
        o.step(o.cfl_dt())
        tots.append(o.conserved_totals())
        divs.append(o.div_b_norm())
    c1, b1, _ = o.get_state()
    return dict(cons=cons, bface=bface, tot0=tot0, abs0=abs0, tots=tots, div0=div0, divs=divs, c1=c1, b1=b1)


def test_conservation(smooth_run):
    r = smooth_run
    for t in r["tots"]:
        assert np.all(np.abs(t - r["tot0"]) <= 1e-14 * r["abs0"]), (t - r["tot0"]) / r["abs0"]
    # the state did change
    assert np.abs(r["c1"] - r["cons"]).max() > 1e-3


def test_div_b_round_off(smooth_run):
    r = smooth_run
    B = np.abs(r["bface"]).max()
    assert r["div0"][0] < 1e-13 * B * 12
    for linf, l2 in r["divs"]:
        assert linf < 1e-12
        assert linf < 1e-13 * B * 12


# ------------------------------------------------------------------ 1-D <-> 3-D


def smooth_1d_state(nx, seed=3):
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / nx
    ph = rng.uniform(0, 2 * np.pi, 8)
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * x + ph[0])
    v = np.stack([0.3 * np.sin(2 * np.pi * x + ph[1]), 0.2 * np.cos(2 * np.pi * x + ph[2]),
                  -0.25 * np.sin(4 * np.pi * x + ph[3])])
    By = 0.8 + 0.3 * np.cos(2 * np.pi * x + ph[4])
    Bz = -0.4 + 0.2 * np.sin(2 * np.pi * x + ph[5])
    Bx = 0.9
    P = 0.6 * (1.0 + 0.2 * np.sin(2 * np.pi * x + ph[6]))
    E = P / (G - 1) + 0.5 * rho * np.sum(v * v, axis=0) + 0.5 * (Bx * Bx + By * By + Bz * Bz)
    u = np.stack([rho, rho * v[0], rho * v[1], rho * v[2], By, Bz, E])
    return u, Bx


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_one_d_equivalence(axis):
    """Grid-aligned 3-D + CT equals the 1-D program (Sec. 3.1.1 vs 3.1.3).
    The 1-D frame (n, t1, t2) is mapped onto the cyclic lab frame of `axis`."""
    nx = 20
    u, Bx = smooth_1d_state(nx)
    h = 1.0 / nx
    lab = [axis, (axis + 1) % 3, (axis + 2) % 3]       # lab index of (n, t1, t2)
    shape = [3, 3, 3]
    shape[axis] = nx
    nxs, nys, nzs = shape

    def to3d(line):
        arr = np.empty((nzs, nys, nxs))
        idx = [None, None, None]
        view = line.reshape([nx if a == axis else 1 for a in (2, 1, 0)])
        arr[...] = view
        return arr

    cons = np.empty((5, nzs, nys, nxs))
    bface = np.empty((3, nzs, nys, nxs))
    cons[0] = to3d(u[0])
    for t in range(3):
        cons[1 + lab[t]] = to3d(u[1 + t])
    cons[4] = to3d(u[6])
    bface[lab[0]] = Bx
    bface[lab[1]] = to3d(u[4])
    bface[lab[2]] = to3d(u[5])
    dx = [0.25, 0.25, 0.25]
    dx[axis] = h
    o = O.Oracle(tuple(shape), tuple(dx))
    o.set_state(cons, bface)
    dt = 0.8 * h / 3.0
    for _ in range(2):
        o.step(dt)
        u = O.step1d(u, h, Bx, dt)
    c1, b1, bc1 = o.get_state()
    scale = np.abs(u).max()
    line = lambda a: np.moveaxis(a, 2 - axis, -1).reshape(-1, nx)
    exp = {0: u[0], 1 + lab[0]: u[1], 1 + lab[1]: u[2], 1 + lab[2]: u[3], 4: u[6]}
    for f, ref in exp.items():
        got = line(c1[f])
        assert np.abs(got - ref).max() <= 1e-13 * scale, (f, np.abs(got - ref).max())
    assert np.abs(line(b1[lab[1]]) - u[4]).max() <= 1e-13 * scale
    assert np.abs(line(b1[lab[2]]) - u[5]).max() <= 1e-13 * scale
    assert np.abs(b1[lab[0]] - Bx).max() <= 1e-15


# ------------------------------------------------------------------ axis relabelling


def test_cyclic_axis_equivariance():
    shape = (10, 8, 6)
    cons, bface = I.random_smooth_state(shape, seed=9)
    dx = (1 / 10, 1 / 8, 1 / 6)
    o = O.Oracle(shape, dx)
    o.set_state(cons, bface)
    dt = 0.5 * o.cfl_dt()
    o.step(dt)
    c1, b1, _ = o.get_state()

    # new axes (x', y', z') = (y, z, x):  A'[z', y', x'] = A[x', ... ] -> transpose (2, 0, 1)
    T = lambda a: np.ascontiguousarray(np.transpose(a, (2, 0, 1)))
    cons_p = np.stack([T(cons[0]), T(cons[2]), T(cons[3]), T(cons[1]), T(cons[4])])
    bface_p = np.stack([T(bface[1]), T(bface[2]), T(bface[0])])
    shape_p = (shape[1], shape[2], shape[0])
    op = O.Oracle(shape_p, (dx[1], dx[2], dx[0]))
    op.set_state(cons_p, bface_p)
    op.step(dt)
    cp, bp, _ = op.get_state()
    exp_c = np.stack([T(c1[0]), T(c1[2]), T(c1[3]), T(c1[1]), T(c1[4])])
    exp_b = np.stack([T(b1[1]), T(b1[2]), T(b1[0])])
    scale = state_scale(cons, bface)
    assert np.abs(cp - exp_c).max() <= 1e-14 * scale
    assert np.abs(bp - exp_b).max() <= 1e-14 * scale


# ------------------------------------------------------------------ convergence


def l1_error(c1, b1, c0, b0):
    """Geometric L1 norm over the state-vector components (Sec. 4)."""
    n = c0[0].size
    comps = [np.abs(c1[f] - c0[f]).sum() / n for f in range(5)] + \
            [np.abs(b1[f] - b0[f]).sum() / n for f in range(3)]
    return float(np.sqrt(np.sum(np.square(comps))))


def run_period(shape, L, cons, bface, T, cfg, cfl=0.8):
    dx = tuple(L[a] / shape[a] for a in range(3))
    o = O.Oracle(shape, dx, cfg)
    o.set_state(cons, bface)
    dt = cfl / 0.8 * o.cfl_dt()
    nsteps = int(np.ceil(T / dt))
    dt = T / nsteps
    for _ in range(nsteps):
        o.step(dt)
    c1, b1, _ = o.get_state()
    return l1_error(c1, b1, cons, bface)


def slopes(Ns, errs):
    return [np.log(errs[i] / errs[i + 1]) / np.log(Ns[i + 1] / Ns[i]) for i in range(len(Ns) - 1)]


def test_convergence_1d_fast_wave():
    """1-D fast magnetosonic wave, one period, WENO5-Z: fifth order (Sec.
    4.1).  CFL 0.4 keeps RK4's fourth-order time error below the spatial
    error; N = 128 would reach the A0^2 wave-steepening floor (~5e-13)."""
    cfg = O.make_config(weno_variant=O.WENO_Z)
    lam, vecs = I.linear_mhd_modes(1.0, 0.0, 1.0, np.sqrt(2.0), 0.5, 1.0 / G)
    dQ = vecs[6]
    cf = lam[6]
    Ns = [16, 32, 64]
    errs = []
    for N in Ns:
        x = (np.arange(N) + 0.5) / N
        s = np.sin(2 * np.pi * x)
        A0 = 1e-6
        bg = np.array([1.0, 0.0, 0.0, 0.0, np.sqrt(2.0), 0.5,
                       (1.0 / G) / (G - 1) + 0.5 * (1 + 2 + 0.25)])
        u0 = bg[:, None] + A0 * dQ[:, None] * s[None, :]
        u = u0.copy()
        dt = 0.4 * (1.0 / N) / cf
        T = 1.0 / cf
        n = int(np.ceil(T / dt))
        for _ in range(n):
            u = O.step1d(u, 1.0 / N, 1.0, T / n, cfg)
        errs.append(np.sqrt(np.sum(np.square(np.abs(u - u0).sum(axis=1) / N))))
    sl = slopes(Ns, errs)
    assert min(sl) > 4.5, (errs, sl)


def oblique_case(N, mode, v_par):
    shape = (N, N, 1)
    L = (1.0, 1.0, 1.0)
    Bw = (1.0, np.sqrt(2.0), 0.5)
    lam, vecs = I.linear_mhd_modes(1.0, v_par, *Bw, 1.0 / G)
    dQ = vecs[mode]
    cons, bface = I.plane_wave_state(shape, L, (1, 1, 0), 1.0, (v_par, 0.0, 0.0), Bw, 1.0 / G, dQ, 1e-6)
    k = 2 * np.pi * np.sqrt(2.0)
    T = (2 * np.pi / k) / abs(lam[mode])
    return shape, L, cons, bface, T


@pytest.mark.slow
def test_convergence_oblique_entropy_wave():
    """Entropy wave (v_par = 1) along (1,1,0): fifth order in L1 (Sec. 4.1:
    the entropy mode carries no field fluctuation)."""
    cfg = O.make_config(weno_variant=O.WENO_Z)
    Ns = [8, 16, 32]
    errs = []
    for N in Ns:
        shape, L, cons, bface, T = oblique_case(N, 3, 1.0)
        errs.append(run_period(shape, L, cons, bface, T, cfg))
    sl = slopes(Ns, errs)
    assert sl[-1] > 4.5, (errs, sl)


@pytest.mark.slow
def test_convergence_oblique_fast_wave():
    """Fast wave along (1,1,0): second order in L1 (the CT update is second
    order, Sec. 4.1)."""
    cfg = O.make_config(weno_variant=O.WENO_Z)
    Ns = [8, 16, 32]
    errs = []
    for N in Ns:
        shape, L, cons, bface, T = oblique_case(N, 6, 0.0)
        errs.append(run_period(shape, L, cons, bface, T, cfg))
    sl = slopes(Ns, errs)
    assert 1.7 < sl[-1] < 3.5, (errs, sl)


# ------------------------------------------------------------------ CFL speeds


def test_max_signal_speed_is_jacobian_spectral_radius():
    """S_d = max(|v_d| + c_f^d) (Eq. cfl); on a uniform state c_f^d is the
    largest |eigenvalue - v_d| of the flux Jacobian along d."""
    from test_oracle_eigen import complex_step_jacobian, prim_to_u
    rho, v, B, P = 1.3, np.array([0.4, -0.7, 0.2]), np.array([0.9, 1.4, -0.6]), 0.7
    shape = (4, 4, 4)
    cons, bface = I.uniform_state(shape, rho=rho, v=tuple(v), B=tuple(B), P=P)
    dx = (0.1, 0.2, 0.3)
    o = O.Oracle(shape, dx)
    o.set_state(cons, bface)
    S = o.max_signal_speed()
    for d in range(3):
        ax = [d, (d + 1) % 3, (d + 2) % 3]
        w = np.array([rho, v[ax[0]], v[ax[1]], v[ax[2]], B[ax[0]], B[ax[1]], B[ax[2]], P])
        ev = np.linalg.eigvals(complex_step_jacobian(prim_to_u(w), w[4])).real
        np.testing.assert_allclose(S[d], np.abs(ev).max(), rtol=1e-12)
    np.testing.assert_allclose(o.cfl_dt(), 0.8 / sum(S[d] / dx[d] for d in range(3)), rtol=1e-15)


def test_worked_example_fast_speed():
    """At the Sec. 4.1 background the fast speed along x is exactly 2."""
    shape = (4, 4, 4)
    cons, bface = I.uniform_state(shape, rho=1.0, B=(1.0, np.sqrt(2.0), 0.5), P=1.0 / G)
    o = O.Oracle(shape, 0.25)
    o.set_state(cons, bface)
    assert abs(o.max_signal_speed()[0] - 2.0) < 1e-15


def test_nonphysical_state_is_reported():
    shape = (6, 4, 4)
    cons, bface = I.uniform_state(shape, rho=1.0, B=(0.5, 0.0, 0.0), P=1.0)
    cons[4, 0, 0, 2] = 0.01          # E below the magnetic energy: P < 0
    o = O.Oracle(shape, 0.25)
    o.set_state(cons, bface)
    with pytest.raises(O.OracleError):
        o.step(1e-3)
    assert o.status()[1] == 1
