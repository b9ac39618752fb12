"""Parity at the benchmark's full size and at the largest configuration,
and on degenerate grids, through the C ABI with the library's own launch
configuration (the one bench.py times).

* 256^3 turbulence (the benchmark input): one FP64 step equals the oracle's
  step on every cell to 1e-12 of the state scale; the FP32-bulk step is
  within float rounding of it.
* 512^3 (the largest configuration, 134M cells): FP32-bulk against FP64 on
  the GPU, conservation and div b (properties that hold at any size; the
  oracle is not run at this size).
* grids with one or more axes of length 1, 2 or 3 (shorter than the
  stencil): FP64 equals the oracle.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1812_04278_gb300 import build
    build.build()
    oracle.build()
    from paper_1812_04278_gb300 import inputs, w5ct
    return dict(torch=torch, O=oracle, I=inputs, W=w5ct)


def solver(env, shape, dx, precision):
    W, torch = env["W"], env["torch"]
    return W.Solver(shape, dx, W.make_config(precision=precision), stream=torch.cuda.current_stream().cuda_stream)


def rel_state(a, b, scale):
    return max(np.abs(a[0] - b[0]).max(), np.abs(a[1] - b[1]).max()) / scale


def test_256_cubed_one_step_fp64_equals_oracle(env):
    I, O, torch = env["I"], env["O"], env["torch"]
    n = 256
    cons, bface = I.turbulent_state(n, seed=1812, seed_b=1813, mach=1.0, beta=1.0, dB_frac=0.1, kmin=2, kmax=32)
    S = max(np.abs(cons).max(), np.abs(bface).max())
    o = O.Oracle((n, n, n), 1.0 / n, O.make_config(weno_variant=O.WENO_Z))
    o.set_state(cons, bface)
    dt = o.cfl_dt()
    cons_d, bface_d = torch.from_numpy(cons).cuda(), torch.from_numpy(bface).cuda()
    g = solver(env, (n, n, n), 1.0 / n, 0)
    g.set_state(cons_d, bface_d)
    assert abs(g.cfl_dt() - dt) <= 1e-14 * dt
    g.step(dt)
    gc, gb, _ = g.get_state()
    g.close()
    o.step(dt)
    oc, ob, _ = o.get_state()
    del o
    err = rel_state((gc, gb), (oc, ob), S)
    assert err <= 1e-12, err
    # FP32-bulk, same input and dt: float rounding of the same step
    f = solver(env, (n, n, n), 1.0 / n, 1)
    f.set_state(cons_d, bface_d)
    f.step(dt)
    fc, fb, _ = f.get_state()
    linf, _ = f.div_b_norm()
    f.close()
    assert rel_state((fc, fb), (oc, ob), S) <= 1e-5
    assert linf < 1e-12


def test_512_cubed_fp32_bulk_properties(env):
    I, torch = env["I"], env["torch"]
    n = 512
    cons, bface = I.analytic_smooth_state((n, n, n), seed=5)
    S = max(np.abs(cons).max(), np.abs(bface).max())
    dv = 1.0 / n ** 3
    absint = np.array([np.abs(cons[f]).sum() for f in range(5)] + [np.abs(bface[f]).sum() for f in range(3)]) * dv
    cons_d, bface_d = torch.from_numpy(cons).cuda(), torch.from_numpy(bface).cuda()
    del cons, bface
    f = solver(env, (n, n, n), 1.0 / n, 1)
    f.set_state(cons_d, bface_d)
    tot0 = f.conserved_totals()
    dt = f.cfl_dt()
    f.step(dt)
    tot1 = f.conserved_totals()
    linf, _ = f.div_b_norm()
    fc = torch.empty_like(cons_d)
    fb = torch.empty_like(bface_d)
    env["W"].w5ct_get_state(f.ctx, fc, fb, None, 1)
    f.close()
    assert linf < 1e-12
    assert np.all(np.abs(tot1 - tot0) <= 1e-10 * absint), (tot1 - tot0) / absint
    g = solver(env, (n, n, n), 1.0 / n, 0)
    g.set_state(cons_d, bface_d)
    g.step(dt)
    gc = torch.empty_like(cons_d)
    gb = torch.empty_like(bface_d)
    env["W"].w5ct_get_state(g.ctx, gc, gb, None, 1)
    tg = g.conserved_totals()
    g.close()
    assert np.all(np.abs(tg - tot0) <= 1e-13 * absint)
    err = max((fc - gc).abs().max().item(), (fb - gb).abs().max().item()) / S
    assert err <= 1e-5, err


@pytest.mark.parametrize("shape", [(1, 8, 8), (16, 1, 1), (1, 1, 1), (2, 3, 1), (7, 2, 5)])
def test_degenerate_grids_fp64_equal_oracle(env, shape):
    I, O, torch = env["I"], env["O"], env["torch"]
    dx = tuple(1.0 / s for s in shape)
    cons, bface = I.analytic_smooth_state(shape, seed=sum(shape))
    S = max(np.abs(cons).max(), np.abs(bface).max())
    o = O.Oracle(shape, dx)
    o.set_state(cons, bface)
    dt = o.cfl_dt()
    g = solver(env, shape, dx, 0)
    g.set_state(torch.from_numpy(cons).cuda(), torch.from_numpy(bface).cuda())
    g.step(dt)
    o.step(dt)
    gc, gb, _ = g.get_state()
    oc, ob, _ = o.get_state()
    g.close()
    assert rel_state((gc, gb), (oc, ob), S) <= 1e-12
