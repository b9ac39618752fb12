"""Oracle pins for the face -> centre field interpolation (Sec. 2.3) and
the floors (a reading: they act inside primitive recovery only).  CPU only.

* The cell field is (9 (b_{i-1/2} + b_{i+1/2}) - (b_{i-3/2} + b_{i+3/2})) / 16
  along each face direction: exact for cubic polynomials at the cell
  centre, fourth order for smooth fields.
* With floors on, a uniform state whose pressure lies below the floor is a
  free-stream state all the same (the floors change the primitives the
  fluxes see, never the conserved state), the floor hits are counted, and
  the signal speed is the closed-form fast speed at the floored pressure.
"""
import numpy as np
import pytest

import oracle
from paper_1812_04278_gb300 import inputs

GAMMA = 5.0 / 3.0


def cubic(x):
    return 0.3 - 1.2 * x + 2.5 * x ** 2 - 1.7 * x ** 3


def face_fields(shape, fx, fy, fz):
    """b_x, b_y, b_z on the forward faces, each a function of its own
    coordinate only (faces at (i + 1) dx, cell centres at (i + 1/2) dx)."""
    nx, ny, nz = shape
    xf = (np.arange(nx) + 1.0) / nx
    yf = (np.arange(ny) + 1.0) / ny
    zf = (np.arange(nz) + 1.0) / nz
    o = np.ones((nz, ny, nx))
    return np.stack([o * fx(xf)[None, None, :], o * fy(yf)[None, :, None], o * fz(zf)[:, None, None]])


def centre_field(shape, bface):
    cons, _ = inputs.uniform_state(shape, rho=1.0, P=1.0)
    o = oracle.Oracle(shape, tuple(1.0 / n for n in shape))
    o.set_state(cons, bface)
    _, _, bcell = o.get_state()
    o.close()
    return bcell


def test_cell_field_is_exact_for_cubics():
    shape = (16, 12, 10)
    bface = face_fields(shape, cubic, lambda y: cubic(1.0 - y), lambda z: cubic(0.5 * z))
    bc = centre_field(shape, bface)
    nx, ny, nz = shape
    xc, yc, zc = (np.arange(nx) + 0.5) / nx, (np.arange(ny) + 0.5) / ny, (np.arange(nz) + 0.5) / nz
    # interior cells: the four faces i-3/2 .. i+3/2 need no periodic wrap
    ex = np.abs(bc[0][:, :, 2:nx - 1] - cubic(xc[2:nx - 1])[None, None, :]).max()
    ey = np.abs(bc[1][:, 2:ny - 1, :] - cubic(1.0 - yc[2:ny - 1])[None, :, None]).max()
    ez = np.abs(bc[2][2:nz - 1, :, :] - cubic(0.5 * zc[2:nz - 1])[:, None, None]).max()
    assert max(ex, ey, ez) < 1e-14, (ex, ey, ez)
    # the wrapped cells see the jump of the non-periodic cubic: not exact
    assert np.abs(bc[0][:, :, 0] - cubic(xc[0])).max() > 1e-3


def test_cell_field_converges_at_fourth_order():
    errs = []
    for n in (8, 16, 32):
        shape = (n, 4, 4)
        k = 2 * np.pi
        bface = face_fields(shape, lambda x: np.sin(k * x), lambda y: np.zeros_like(y), lambda z: np.zeros_like(z))
        bc = centre_field(shape, bface)
        xc = (np.arange(n) + 0.5) / n
        errs.append(np.abs(bc[0][0, 0, :] - np.sin(k * xc)).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 3.8), (errs, orders)


def fast_speed(rho, P, Bn, Bt2):
    """c_f from the root formula (reading of Eqs. slow/fast)."""
    cs2, ca2, bt2 = GAMMA * P / rho, Bn * Bn / rho, Bt2 / rho
    s = cs2 + ca2 + bt2
    return np.sqrt(0.5 * (s + np.sqrt(s * s - 4.0 * cs2 * ca2)))


def test_floors_touch_only_the_primitives():
    shape = (8, 6, 4)
    v, B, P, p_min = (0.3, -0.2, 0.1), (0.5, 0.2, -0.1), 1e-10, 1e-8
    cons, bface = inputs.uniform_state(shape, rho=1.0, v=v, B=B, P=P)
    o = oracle.Oracle(shape, tuple(1.0 / n for n in shape),
                      oracle.make_config(floors=1, rho_min=1e-8, p_min=p_min))
    o.set_state(cons, bface)
    S = o.max_signal_speed()
    for d in range(3):
        Bt2 = sum(B[e] ** 2 for e in range(3) if e != d)
        floored = abs(v[d]) + fast_speed(1.0, p_min, B[d], Bt2)
        raw = abs(v[d]) + fast_speed(1.0, P, B[d], Bt2)
        assert abs(S[d] - floored) <= 1e-12 * floored, (d, S[d], floored)
        assert abs(S[d] - raw) > 1e-9 * raw        # the floored pressure, not the stored one
    dt = o.cfl_dt()
    o.step(dt)
    c, b, _ = o.get_state()
    hits, bad = o.status()
    o.close()
    assert bad == 0 and hits > 0
    assert np.abs(c - cons).max() <= 1e-14 * np.abs(cons).max()
    assert np.abs(b - bface).max() <= 1e-14 * np.abs(bface).max()


def mirror_x(cons, bface):
    """The state reflected in x (x -> L - x): rho, E, m_y, m_z, b_y, b_z keep
    their values at the mirrored cell, m_x and b_x change sign, and the
    forward x face i + 1/2 maps to the face (n - 2 - i) + 1/2."""
    nx = cons.shape[3]
    c = cons[:, :, :, ::-1].copy()
    c[1] = -c[1]
    b = np.empty_like(bface)
    b[0] = -bface[0][:, :, (nx - 2 - np.arange(nx)) % nx]
    b[1] = bface[1][:, :, ::-1]
    b[2] = bface[2][:, :, ::-1]
    return c, b


@pytest.mark.parametrize("variant", [oracle.WENO_JS, oracle.WENO_Z])
def test_step_commutes_with_reflection(variant):
    """Ideal MHD is invariant under x -> -x with v_x -> -v_x and B_x -> -B_x,
    and the scheme treats the two WENO sides, the mode pairs and the two
    cells of every face alike: three steps of the reflected state, reflected
    back, equal three steps of the state to rounding.  (With the cyclic
    relabelling this covers the y and z reflections too.)"""
    shape = (16, 8, 6)
    dx = tuple(1.0 / n for n in shape)
    cons, bface = inputs.random_smooth_state(shape, seed=77)
    a = oracle.Oracle(shape, dx, oracle.make_config(weno_variant=variant))
    b = oracle.Oracle(shape, dx, oracle.make_config(weno_variant=variant))
    a.set_state(cons, bface)
    b.set_state(*mirror_x(cons, bface))
    dt = a.cfl_dt()
    assert b.cfl_dt() == dt
    for _ in range(3):
        a.step(dt)
        b.step(dt)
    ca, ba, _ = a.get_state()
    rc, rb = mirror_x(*b.get_state()[:2])
    a.close()
    b.close()
    S = max(np.abs(ca).max(), np.abs(ba).max())
    assert np.abs(rc - ca).max() <= 1e-14 * S
    assert np.abs(rb - ba).max() <= 1e-14 * S


def test_step_commutes_with_density_scaling():
    """Ideal MHD is invariant under rho, P, E -> 4x and B -> 2x with v
    unchanged (every wave speed stays the same), and so is the scheme with
    WENO-Z, whose epsilon_Z = 1e-40 lies below rounding: with factors that
    are powers of two every operation scales exactly, so the scaled state
    steps to exactly the scaled result.  A wrong power of rho anywhere (the
    sqrt(rho) of the Alfven and magnetosonic eigenvectors, the B / sqrt(rho)
    of c_A) breaks this."""
    shape = (12, 8, 6)
    dx = tuple(1.0 / n for n in shape)
    cons, bface = inputs.random_smooth_state(shape, seed=91)
    a = oracle.Oracle(shape, dx, oracle.make_config(weno_variant=oracle.WENO_Z))
    b = oracle.Oracle(shape, dx, oracle.make_config(weno_variant=oracle.WENO_Z))
    a.set_state(cons, bface)
    b.set_state(4.0 * cons, 2.0 * bface)
    dt = a.cfl_dt()
    assert b.cfl_dt() == dt
    for _ in range(3):
        a.step(dt)
        b.step(dt)
    ca, ba, _ = a.get_state()
    cb, bb, _ = b.get_state()
    a.close()
    b.close()
    assert np.array_equal(cb, 4.0 * ca)
    assert np.array_equal(bb, 2.0 * ba)


def test_step_commutes_with_velocity_scaling():
    """The other unit change of ideal MHD: v, B -> 2x, P, E -> 4x (rho
    fixed) is the same flow run twice as fast, so the CFL step halves and a
    step of dt/2 of the scaled state is exactly the scaled step of dt (WENO-Z,
    powers of two).  Together with the density scaling this pins how dt
    enters the stages and the relative dimensions of every v, B and P term."""
    shape = (12, 8, 6)
    dx = tuple(1.0 / n for n in shape)
    cons, bface = inputs.random_smooth_state(shape, seed=93)
    sc = np.array([1.0, 2.0, 2.0, 2.0, 4.0])[:, None, None, None]
    a = oracle.Oracle(shape, dx, oracle.make_config(weno_variant=oracle.WENO_Z))
    b = oracle.Oracle(shape, dx, oracle.make_config(weno_variant=oracle.WENO_Z))
    a.set_state(cons, bface)
    b.set_state(sc * cons, 2.0 * bface)
    dt = a.cfl_dt()
    assert b.cfl_dt() == 0.5 * dt
    for _ in range(3):
        a.step(dt)
        b.step(0.5 * dt)
    ca, ba, _ = a.get_state()
    cb, bb, _ = b.get_state()
    a.close()
    b.close()
    assert np.array_equal(cb, sc * ca)
    assert np.array_equal(bb, 2.0 * ba)


def swap_xy(cons, bface):
    """The state with x and y exchanged (v_x <-> v_y, b_x <-> b_y); nx = ny."""
    c = np.ascontiguousarray(cons.transpose(0, 1, 3, 2))
    c[[1, 2]] = c[[2, 1]]
    b = np.ascontiguousarray(bface.transpose(0, 1, 3, 2))
    b[[0, 1]] = b[[1, 0]]
    return c, b


@pytest.mark.parametrize("variant", [oracle.WENO_JS, oracle.WENO_Z])
def test_step_commutes_with_the_xy_swap(variant):
    """Exchanging x and y is a symmetry of ideal MHD; the paper's implosion
    test (Sec. 4.7) relies on the scheme keeping a state symmetric about
    x = y.  The swap is an odd permutation, so the cyclic relabelling does
    not cover it: it exchanges the transverse ordering (t1, t2) of the sweep
    frames and the signs of the Alfven eigenvectors and of the EMFs.  Three
    steps of the swapped state, swapped back, equal three steps of the state
    to rounding."""
    shape = (12, 12, 8)
    dx = tuple(1.0 / n for n in shape)
    cons, bface = inputs.random_smooth_state(shape, seed=71)
    a = oracle.Oracle(shape, dx, oracle.make_config(weno_variant=variant))
    b = oracle.Oracle(shape, dx, oracle.make_config(weno_variant=variant))
    a.set_state(cons, bface)
    b.set_state(*swap_xy(cons, bface))
    dt = a.cfl_dt()
    assert b.cfl_dt() == dt
    for _ in range(3):
        a.step(dt)
        b.step(dt)
    ca, ba, _ = a.get_state()
    rc, rb = swap_xy(*b.get_state()[:2])
    a.close()
    b.close()
    S = max(np.abs(ca).max(), np.abs(ba).max())
    assert np.abs(rc - ca).max() <= 1e-14 * S
    assert np.abs(rb - ba).max() <= 1e-14 * S
