"""Several patches advanced by one context (batched launches over a tile
table, per-patch dt, graph replay), through the C ABI.

Every patch of a batch runs the same per-cell and per-face arithmetic as a
context holding that patch alone, so the batched results must equal the
single-patch ones bit for bit; FP64 batches are also checked against the
oracle to 1e-12 per step (the bound of the single-patch parity tests).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL64 = 1e-12

# uneven sizes: ragged x tiles, patches smaller than one tile, ny below the
# stencil width, and one patch spanning several tiles in every direction
SHAPES = [(16, 16, 16), (24, 16, 32), (33, 9, 10), (8, 8, 8), (48, 24, 16), (12, 3, 17)]


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1812_04278_gb300 import build
    build.build()
    from paper_1812_04278_gb300 import inputs, w5ct
    oracle.build()
    return dict(torch=torch, O=oracle, I=inputs, W=w5ct)


def states(env, shapes, seed0):
    I = env["I"]
    return [I.random_smooth_state(sh, seed=seed0 + p) for p, sh in enumerate(shapes)]


def spacings(shapes):
    return [tuple(1.0 / n for n in sh) for sh in shapes]


def make_batch(env, shapes, sts, precision, variant):
    W, torch = env["W"], env["torch"]
    b = W.Batch(shapes, spacings(shapes), W.make_config(precision=precision, weno_variant=variant),
                stream=torch.cuda.current_stream().cuda_stream)
    for p, (cons, bface) in enumerate(sts):
        b.set_state(p, cons, bface)
    return b


def make_single(env, shape, st, precision, variant):
    W, torch = env["W"], env["torch"]
    s = W.Solver(shape, tuple(1.0 / n for n in shape), W.make_config(precision=precision, weno_variant=variant),
                 stream=torch.cuda.current_stream().cuda_stream)
    s.set_state(*st)
    return s


def assert_same(a, b, what):
    for x, y, name in zip(a, b, ("cons", "bface", "bcell")):
        assert np.array_equal(x, y), (what, name, np.abs(x - y).max())


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("variant", [0, 1])
def test_batched_step_equals_single_patches(env, precision, variant):
    sts = states(env, SHAPES, 100 + 10 * precision + variant)
    b = make_batch(env, SHAPES, sts, precision, variant)
    dt = 0.2 * min(1.0 / n for sh in SHAPES for n in sh)
    for _ in range(2):
        b.step(dt)
    for p, sh in enumerate(SHAPES):
        s = make_single(env, sh, sts[p], precision, variant)
        for _ in range(2):
            s.step(dt)
        assert_same(b.get_state(p), s.get_state(), ("patch", p, sh))
        s.close()
    b.close()


@pytest.mark.parametrize("variant", [0, 1])
def test_fp64_batch_matches_oracle(env, variant):
    O = env["O"]
    sts = states(env, SHAPES, 200 + variant)
    b = make_batch(env, SHAPES, sts, 0, variant)
    oras = []
    for p, sh in enumerate(SHAPES):
        o = O.Oracle(sh, tuple(1.0 / n for n in sh), O.make_config(weno_variant=variant))
        o.set_state(*sts[p])
        oras.append(o)
    dts = [o.cfl_dt() for o in oras]
    torch = env["torch"]
    dts_dev = torch.tensor(dts, dtype=torch.float64, device="cuda")
    b.step_dev(dts_dev)
    for p, o in enumerate(oras):
        o.step(dts[p])
        gc, gb, _ = b.get_state(p)
        oc, ob, _ = o.get_state()
        S = max(np.abs(oc).max(), np.abs(ob).max())
        err = max(np.abs(gc - oc).max(), np.abs(gb - ob).max()) / S
        assert err <= TOL64, (p, SHAPES[p], err)
    b.close()


@pytest.mark.parametrize("schedule", [1, 2])
@pytest.mark.parametrize("variant", [0, 1])
def test_fp64_persistent_and_fused_schedules_match_oracle(env, schedule, variant):
    """Schedules 1 (persistent sweeps) and 2 (the whole step in one persistent
    launch) against the oracle directly: every patch, after each of two steps
    of the oracle's own CFL dt, within 1e-12 per step of the state scale."""
    O, torch = env["O"], env["torch"]
    sts = states(env, SHAPES, 1300 + 10 * schedule + variant)
    b = make_batch(env, SHAPES, sts, 0, variant)
    b.set_schedule(schedule)
    assert b.schedule() == schedule
    oras = []
    for p, sh in enumerate(SHAPES):
        o = O.Oracle(sh, tuple(1.0 / n for n in sh), O.make_config(weno_variant=variant))
        o.set_state(*sts[p])
        oras.append(o)
    for k in range(2):
        dts = [o.cfl_dt() for o in oras]
        b.step_dev(torch.tensor(dts, dtype=torch.float64, device="cuda"))
        for p, o in enumerate(oras):
            o.step(dts[p])
            gc, gb, _ = b.get_state(p)
            oc, ob, _ = o.get_state()
            S = max(np.abs(oc).max(), np.abs(ob).max())
            err = max(np.abs(gc - oc).max(), np.abs(gb - ob).max()) / S
            assert err <= TOL64 * (k + 1), (k, p, SHAPES[p], err)
    assert b.status()[1] == 0
    b.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_per_patch_cfl_dt(env, precision):
    """step_cfl gives every patch the dt its own state fixes (Eq. cfl), equal
    to the dt a context of that patch alone computes."""
    torch = env["torch"]
    sts = states(env, SHAPES, 300 + precision)
    b = make_batch(env, SHAPES, sts, precision, 1)
    dts = torch.zeros(len(SHAPES), dtype=torch.float64, device="cuda")
    b.step_cfl(dts)
    dts_b = dts.cpu().numpy()
    assert len(set(dts_b.tolist())) == len(SHAPES)     # the patches take different dts
    for p, sh in enumerate(SHAPES):
        s = make_single(env, sh, sts[p], precision, 1)
        d1 = torch.zeros(1, dtype=torch.float64, device="cuda")
        s.step_cfl(d1)
        assert d1.item() == dts_b[p], (p, d1.item(), dts_b[p])
        assert_same(b.get_state(p), s.get_state(), ("patch", p, sh))
        s.close()
    b.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_equals_eager_steps(env, precision):
    sts = states(env, SHAPES, 400 + precision)
    a = make_batch(env, SHAPES, sts, precision, 1)
    e = make_batch(env, SHAPES, sts, precision, 1)
    a.step_graph(2)
    a.step_graph(1)           # reuses the captured graph
    for _ in range(3):
        e.step_cfl()
    a.synchronize()
    e.synchronize()
    for p in range(len(SHAPES)):
        assert_same(a.get_state(p), e.get_state(p), ("patch", p))
    assert a.status()[1] == 0 and e.status()[1] == 0       # no non-physical state flagged
    a.close()
    e.close()


def test_batched_diagnostics_are_per_patch(env):
    sts = states(env, SHAPES, 500)
    b = make_batch(env, SHAPES, sts, 0, 1)
    b.step_cfl()
    b.synchronize()
    for p, sh in enumerate(SHAPES):
        s = make_single(env, sh, sts[p], 0, 1)
        s.step_cfl()
        assert np.array_equal(b.max_signal_speed(p), s.max_signal_speed())
        linf_b, l2_b = b.div_b_norm(p)
        linf_s, l2_s = s.div_b_norm()
        assert linf_b == linf_s and abs(l2_b - l2_s) <= 1e-14 * max(l2_s, 1e-300)
        np.testing.assert_allclose(b.conserved_totals(p), s.conserved_totals(), rtol=1e-13, atol=1e-15)
        s.close()
    b.close()


def test_batch_rejects_bad_patch_index(env):
    W = env["W"]
    sts = states(env, SHAPES[:2], 600)
    b = make_batch(env, SHAPES[:2], sts, 0, 1)
    with pytest.raises(W.W5ctError) as e:
        W.w5ct_max_signal_speed(b.ctx, 2)
    assert e.value.code == W.W5CT_ERR_ARG
    b.close()


@pytest.fixture(scope="module")
def single_fp32(env):
    """Two fixed-dt FP32-bulk steps of every patch of SHAPES, one context per
    patch (the reference of the tile-variant tests)."""
    sts = states(env, SHAPES, 700)
    dt = 0.2 * min(1.0 / n for sh in SHAPES for n in sh)
    out = []
    for p, sh in enumerate(SHAPES):
        s = make_single(env, sh, sts[p], 1, 1)
        s.step(dt)
        s.step(dt)
        out.append(s.get_state())
        s.close()
    return sts, dt, out


@pytest.mark.parametrize("mode", [0, 1, 2, 3, -2, -1])
def test_tile_variants_do_not_change_results(env, single_fp32, mode):
    """Every sweep tile shape (forced, the model's choice or the measured
    autotuner's) computes each face with the same arithmetic."""
    W = env["W"]
    sts, dt, ref = single_fp32
    b = make_batch(env, SHAPES, sts, 1, 1)
    b.autotune(mode, 2)
    b.set_schedule(0)          # the schedules agree only to rounding (tested below)
    counts = b.tile_variants()
    assert counts.sum(axis=1).tolist() == [len(SHAPES)] * 3
    if mode >= 0:
        assert counts[:, mode].tolist() == [len(SHAPES)] * 3
    b.step(dt)
    b.step(dt)
    for p in range(len(SHAPES)):
        assert_same(b.get_state(p), ref[p], ("mode", mode, "patch", p))
    assert b.status() == (0, 0)
    b.close()


def test_tile_model_prefers_full_tiles(env):
    W = env["W"]
    shapes = [(64, 64, 64), (16, 16, 16), (24, 24, 24)]
    sts = states(env, shapes, 800)
    b = make_batch(env, shapes, sts, 1, 1)
    assert W.w5ct_tile_variant(b.ctx, 0, 0) == (0, 32, 16)     # 64 = 2 x 32 lanes
    assert W.w5ct_tile_variant(b.ctx, 0, 1)[1] == 16           # 16 lanes, not half of 32
    assert W.w5ct_tile_variant(b.ctx, 0, 2)[1] == 8            # 24 = 3 x 8 lanes
    b.close()


def test_fp64_has_only_the_default_tile(env):
    W = env["W"]
    sts = states(env, SHAPES[:2], 900)
    b = make_batch(env, SHAPES[:2], sts, 0, 1)
    with pytest.raises(W.W5ctError) as e:
        b.autotune(1)
    assert e.value.code == W.W5CT_ERR_ARG
    b.autotune(W.W5CT_TUNE_MEASURE, 1)
    assert b.tile_variants()[:, 0].tolist() == [2, 2, 2]
    b.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("variant", [0, 1])
def test_persistent_schedule_gives_the_same_results(env, single_fp32, precision, variant):
    """The persistent work-queue sweep (schedule 1) computes every face from
    the same source as one launch per axis; the compiler may contract a few
    operations differently in the fused kernel, so the states agree to
    rounding (1e-13 of the state scale after four steps, eager and replayed
    from a graph, several tile variants in use)."""
    sts = states(env, SHAPES, 1000 + 10 * precision + variant)
    a = make_batch(env, SHAPES, sts, precision, variant)
    b = make_batch(env, SHAPES, sts, precision, variant)
    b.set_schedule(1)
    assert b.schedule() == 1
    for _ in range(2):
        a.step_cfl()
        b.step_cfl()
    b.step_graph(2)
    a.step_graph(2)
    a.synchronize()
    b.synchronize()
    tol = 1e-13 if precision == 0 else 1e-5
    for p in range(len(SHAPES)):
        for x, y in zip(a.get_state(p), b.get_state(p)):
            assert np.abs(x - y).max() <= tol * np.abs(x).max(), ("patch", p)
    assert b.status()[1] == 0
    a.close()
    b.close()


def test_persistent_schedule_needs_a_batch(env):
    W, torch = env["W"], env["torch"]
    s = W.Solver((8, 8, 8), 0.125, W.make_config(), stream=torch.cuda.current_stream().cuda_stream)
    for sched in (1, 2):
        with pytest.raises(W.W5ctError) as e:
            W.w5ct_set_sweep_schedule(s.ctx, sched)
        assert e.value.code == W.W5CT_ERR_UNSUPPORTED
    with pytest.raises(W.W5ctError) as e:
        W.w5ct_set_sweep_schedule(s.ctx, 3)
    assert e.value.code == W.W5CT_ERR_ARG
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("variant", [0, 1])
def test_fused_step_agrees_with_launch_per_kernel(env, precision, variant):
    """Schedule 2 (the whole step in one persistent launch over a work queue
    with per-patch dependencies) gives the states and per-patch dts of the
    launch-per-kernel schedule, through every step entry point and a graph
    replay; no wait expires."""
    torch = env["torch"]
    sts = states(env, SHAPES, 1100 + 10 * precision + variant)
    a = make_batch(env, SHAPES, sts, precision, variant)
    b = make_batch(env, SHAPES, sts, precision, variant)
    b.set_schedule(2)
    assert b.schedule() == 2
    da = torch.zeros(len(SHAPES), dtype=torch.float64, device="cuda")
    db = torch.zeros_like(da)
    a.step_cfl(da)
    b.step_cfl(db)
    if precision == 0:
        assert torch.equal(da, db)                 # double maxima and dt: the same operations
    else:
        assert torch.allclose(da, db, rtol=1e-6, atol=0)   # float speeds, contracted per kernel
    dt = 0.1 * min(1.0 / n for sh in SHAPES for n in sh)
    a.step(dt)
    b.step(dt)
    a.step_dev(da)
    b.step_dev(db)
    a.step_graph(2)
    b.step_graph(2)
    a.synchronize()
    b.synchronize()
    tol = 1e-13 if precision == 0 else 1e-5
    for p in range(len(SHAPES)):
        for x, y in zip(a.get_state(p), b.get_state(p)):
            assert np.abs(x - y).max() <= tol * np.abs(x).max(), ("patch", p)
    assert b.status() == a.status()
    a.close()
    b.close()


def test_fused_step_many_small_patches(env):
    """Many patches smaller than one tile: most items of a stage wait on
    others of their patch (the dependency chains of the work queue)."""
    shapes = [(8 + (p % 3) * 4, 6 + (p % 2) * 5, 4 + (p % 4)) for p in range(40)]
    sts = [env["I"].random_smooth_state(sh, seed=1200 + p) for p, sh in enumerate(shapes)]
    a = make_batch(env, shapes, sts, 0, 1)
    b = make_batch(env, shapes, sts, 0, 1)
    b.set_schedule(2)
    for _ in range(3):
        a.step_cfl()
        b.step_cfl()
    a.synchronize()
    b.synchronize()
    for p in range(len(shapes)):
        for x, y in zip(a.get_state(p), b.get_state(p)):
            assert np.abs(x - y).max() <= 1e-13 * np.abs(x).max(), ("patch", p)
    a.close()
    b.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_fused_wait_expiry_reports_timeout(env, precision):
    """A fused-step wait that nothing satisfies (a one-item work list whose
    sweep dependency is never done) ends after its bound: the launch aborts
    and ends on its own, the status reads W5CT_ERR_TIMEOUT, the state is
    untouched, and the context then steps like a fresh one."""
    import time
    W = env["W"]
    sts = states(env, SHAPES, 1300 + precision)
    a = make_batch(env, SHAPES, sts, precision, 1)
    b = make_batch(env, SHAPES, sts, precision, 1)
    before = [b.get_state(p) for p in range(len(SHAPES))]
    t0 = time.perf_counter()
    status = W.w5ct_fused_wait_check(b.ctx, 1000)       # 1000 sleeps of 256 ns
    elapsed = time.perf_counter() - t0
    assert status == W.W5CT_ERR_TIMEOUT
    assert elapsed < 5.0
    for p in range(len(SHAPES)):
        for x, y in zip(before[p], b.get_state(p)):
            assert np.array_equal(x, y), ("state changed by the aborted launch", p)
    assert b.status()[1] == 0                           # flag restored
    b.set_schedule(2)
    for _ in range(2):
        a.step_cfl()
        b.step_cfl()
    a.synchronize()
    b.synchronize()
    tol = 1e-13 if precision == 0 else 1e-5
    for p in range(len(SHAPES)):
        for x, y in zip(a.get_state(p), b.get_state(p)):
            assert np.abs(x - y).max() <= tol * np.abs(x).max(), ("patch", p)
    with pytest.raises(Exception):
        W.w5ct_fused_wait_check(b.ctx, 0)                # bound out of range
    a.close()
    b.close()
