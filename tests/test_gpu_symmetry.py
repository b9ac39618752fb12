"""Symmetries of ideal MHD that the scheme keeps, on the FP64 GPU path
(libw5ct through the C ABI): the same pins the oracle satisfies
(tests/test_oracle_fields.py), now for the CUDA kernels.

* x reflection (v_x, B_x -> -v_x, -B_x, forward faces remapped) and the
  x <-> y swap (the symmetry about x = y of the implosion test, Sec. 4.7):
  three steps of the transformed state, transformed back, equal three steps
  of the state to rounding (the kernels contract operations into FMAs, so
  the bar is 1e-13 of the state scale against the oracle's 1e-14);
* the density scaling (rho, P, E -> 4x, B -> 2x) and the time-unit scaling
  (v, B -> 2x, P, E -> 4x, dt -> dt/2): with powers of two every operation,
  the Newton-Raphson reciprocal included, scales exactly, so the steps agree
  bit for bit (WENO-Z, whose eps_Z lies below rounding).
"""
import numpy as np
import pytest

from test_oracle_fields import mirror_x, swap_xy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_04278_gb300 import build
    build.build()
    from paper_1812_04278_gb300 import inputs, w5ct
    return torch, inputs, w5ct


def run(env, shape, cons, bface, dt, nsteps=3, variant=1):
    torch, I, W = env
    s = W.Solver(shape, tuple(1.0 / n for n in shape), W.make_config(weno_variant=variant),
                 stream=torch.cuda.current_stream().cuda_stream)
    s.set_state(cons, bface)
    for _ in range(nsteps):
        s.step(dt)
    c, b, _ = s.get_state()
    s.close()
    return c, b


def cfl(env, shape, cons, bface):
    torch, I, W = env
    s = W.Solver(shape, tuple(1.0 / n for n in shape), W.make_config(), stream=torch.cuda.current_stream().cuda_stream)
    s.set_state(cons, bface)
    dt = W.w5ct_cfl_dt(s.ctx)
    s.close()
    return dt


@pytest.mark.parametrize("variant", [0, 1])
def test_gpu_step_commutes_with_reflection(env, variant):
    shape = (16, 8, 6)
    cons, bface = env[1].random_smooth_state(shape, seed=77)
    dt = cfl(env, shape, cons, bface)
    ca, ba = run(env, shape, cons, bface, dt, variant=variant)
    rc, rb = mirror_x(*run(env, shape, *mirror_x(cons, bface), dt, variant=variant))
    S = max(np.abs(ca).max(), np.abs(ba).max())
    assert np.abs(rc - ca).max() <= 1e-13 * S
    assert np.abs(rb - ba).max() <= 1e-13 * S


@pytest.mark.parametrize("variant", [0, 1])
def test_gpu_step_commutes_with_the_xy_swap(env, variant):
    shape = (12, 12, 8)
    cons, bface = env[1].random_smooth_state(shape, seed=71)
    dt = cfl(env, shape, cons, bface)
    ca, ba = run(env, shape, cons, bface, dt, variant=variant)
    rc, rb = swap_xy(*run(env, shape, *swap_xy(cons, bface), dt, variant=variant))
    S = max(np.abs(ca).max(), np.abs(ba).max())
    assert np.abs(rc - ca).max() <= 1e-13 * S
    assert np.abs(rb - ba).max() <= 1e-13 * S


def test_gpu_step_commutes_with_density_scaling(env):
    shape = (12, 8, 6)
    cons, bface = env[1].random_smooth_state(shape, seed=91)
    dt = cfl(env, shape, cons, bface)
    assert cfl(env, shape, 4.0 * cons, 2.0 * bface) == dt
    ca, ba = run(env, shape, cons, bface, dt)
    cb, bb = run(env, shape, 4.0 * cons, 2.0 * bface, dt)
    assert np.array_equal(cb, 4.0 * ca)
    assert np.array_equal(bb, 2.0 * ba)


def test_gpu_step_commutes_with_velocity_scaling(env):
    shape = (12, 8, 6)
    cons, bface = env[1].random_smooth_state(shape, seed=93)
    sc = np.array([1.0, 2.0, 2.0, 2.0, 4.0])[:, None, None, None]
    dt = cfl(env, shape, cons, bface)
    assert cfl(env, shape, sc * cons, 2.0 * bface) == 0.5 * dt
    ca, ba = run(env, shape, cons, bface, dt)
    cb, bb = run(env, shape, sc * cons, 2.0 * bface, 0.5 * dt)
    assert np.array_equal(cb, sc * ca)
    assert np.array_equal(bb, 2.0 * ba)
