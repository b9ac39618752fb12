"""Parity at the two largest configurations' full size, in the launch
configuration the benchmark times, on sampled outputs the oracle can compute
(libw5ct through the C ABI).

* The 512^3 magnetised blast in Mach-5 turbulence (WENO-JS, floors on): one
  FP64 step of the whole grid on the GPU.  One step of the scheme reaches
  only a bounded distance -- per RK stage about three cells through the
  flux stencil, two through the face-to-centre interpolation of the field
  and one through the corner EMFs, so under 24 cells for the four stages
  (Secs. 2.1-2.3) -- so the oracle run on a periodic 72^3 sub-box of the
  same cells (same spacing) reproduces the full grid's step exactly in the
  sub-box's central 8^3 cells, 32 cells from its seams.  Four such boxes (at
  the blast centre, across the periodic wrap, and two seeded positions) must
  equal the GPU's step to 1e-12 of the state scale.  dt is fixed (CFL about
  0.45 of the state's fastest signal); nothing of the oracle's input comes
  from the GPU.
* The 512-patch batch (uneven sizes, FP64, floors on): every patch advances
  one step with its own dt from the oracle's CFL condition in one batched
  step; four sampled patches (the smallest, the largest and two seeded ones)
  run whole in the oracle must agree to 1e-12.
"""
import os
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL64 = 1e-12


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


def test_blast_512_cubed_fp64_step_equals_oracle_on_sampled_boxes(env):
    torch, O, I, W = env["torch"], env["O"], env["I"], env["W"]
    n = 512
    cons, bface = I.blast_turbulence_state(n)
    S = max(np.abs(cons).max(), np.abs(bface).max())
    dt = 1.5e-5
    dx = 1.0 / n
    s = W.Solver((n, n, n), dx, W.make_config(precision=W.W5CT_FP64, weno_variant=W.W5CT_WENO_JS, floors=1),
                 stream=torch.cuda.current_stream().cuda_stream)
    cons_d, bface_d = torch.from_numpy(cons).cuda(), torch.from_numpy(bface).cuda()
    s.set_state(cons_d, bface_d)
    s.step(dt)
    gc, gb = torch.empty_like(cons_d), torch.empty_like(bface_d)
    W.w5ct_get_state(s.ctx, gc, gb, None, 1)
    assert s.status()[1] == 0
    s.close()
    del cons_d, bface_d
    core, margin = 8, 32
    sub = core + 2 * margin
    rng = np.random.default_rng(512)
    centres = [(n // 2, n // 2, n // 2), (n - 3, 1, n // 2)] + [tuple(int(v) for v in rng.integers(0, n, 3))
                                                                    for _ in range(2)]
    cfg = O.make_config(weno_variant=O.WENO_JS, floors=1)
    for cx, cy, cz in centres:
        ix, iy, iz = ((c - sub // 2 + np.arange(sub)) % n for c in (cx, cy, cz))
        sel = np.ix_(iz, iy, ix)
        o = O.Oracle((sub, sub, sub), dx, cfg)
        o.set_state(np.ascontiguousarray(cons[(slice(None),) + sel]), np.ascontiguousarray(bface[(slice(None),) + sel]))
        o.step(dt)
        oc, ob, _ = o.get_state()
        o.close()
        k = slice(margin, margin + core)
        gsel = (slice(None),) + tuple(torch.from_numpy(v[k].copy()).cuda() for v in (iz, iy, ix))
        gcc = gc[:, gsel[1][:, None, None], gsel[2][None, :, None], gsel[3][None, None, :]].cpu().numpy()
        gbb = gb[:, gsel[1][:, None, None], gsel[2][None, :, None], gsel[3][None, None, :]].cpu().numpy()
        err = max(np.abs(gcc - oc[:, k, k, k]).max(), np.abs(gbb - ob[:, k, k, k]).max()) / S
        assert err <= TOL64, ((cx, cy, cz), err)


def test_batched_512_patches_fp64_equal_oracle_on_sampled_patches(env):
    torch, O, I, W = env["torch"], env["O"], env["I"], env["W"]
    sys.path.insert(0, ROOT)
    import bench
    specs = I.patch_batch_spec(npatch=512, seed=1803)
    states = bench.batch_states(specs, min(16, os.cpu_count() or 1))
    shapes = [sp["shape"] for sp in specs]
    dxs = [sp["dx"] for sp in specs]
    cfg = O.make_config(floors=1)
    dts = []
    for sh, dx, st in zip(shapes, dxs, states):
        o = O.Oracle(sh, dx, cfg)
        o.set_state(*st)
        dts.append(o.cfl_dt())
        o.close()
    b = W.Batch(shapes, dxs, W.make_config(precision=W.W5CT_FP64, floors=1),
                stream=torch.cuda.current_stream().cuda_stream)
    for p, (c, f) in enumerate(states):
        b.set_state(p, c, f)
    b.step_dev(torch.tensor(dts, dtype=torch.float64, device="cuda"))
    sizes = [int(np.prod(sh)) for sh in shapes]
    rng = np.random.default_rng(1803)
    sample = sorted({int(np.argmin(sizes)), int(np.argmax(sizes))} | {int(v) for v in rng.integers(0, 512, 2)})
    for p in sample:
        o = O.Oracle(shapes[p], dxs[p], cfg)
        o.set_state(*states[p])
        o.step(dts[p])
        oc, ob, _ = o.get_state()
        o.close()
        gc, gb, _ = b.get_state(p)
        S = max(np.abs(oc).max(), np.abs(ob).max())
        err = max(np.abs(gc - oc).max(), np.abs(gb - ob).max()) / S
        assert err <= TOL64, (p, shapes[p], err)
    assert b.status()[1] == 0
    b.close()
