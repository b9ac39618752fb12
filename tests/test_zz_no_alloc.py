"""w5ct_conserved_totals_noalloc: the conserved-totals reduction for callers
that cannot allocate device memory (frameworks that own all device memory,
real-time loops that cannot take an allocation's synchronisation).  Checked
through the C ABI against the regular entry point w5ct_conserved_totals on
two calls in a row with different inputs, so a second call cannot pass on
the first call's leftovers in the shared fixed scratch; and the device's
free memory is the same before and after a call.

The file name sorts last so that pytest collects it after every other test:
a run that stops at the first failure (-x) has then already run the rest of
the suite if this one fails.  Nothing in it depends on the other tests."""
import numpy as np
import pytest

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


def test_noalloc_totals_match_the_context_entry_point(env):
    torch, I, W = env
    shape = (40, 24, 36)            # ragged against the 16384-cell blocks
    dx = (1 / 40, 1 / 24, 1 / 36)
    stream = torch.cuda.current_stream().cuda_stream
    s = W.Solver(shape, dx, W.make_config(), stream=stream)
    for seed in (11, 12):           # two calls in a row, different states
        cons, bface = I.random_smooth_state(shape, seed=seed)
        cons_d = torch.from_numpy(cons).cuda()
        bface_d = torch.from_numpy(bface).cuda()
        s.set_state(cons_d, bface_d)
        ref = W.w5ct_conserved_totals(s.ctx)
        got = W.w5ct_conserved_totals_noalloc(cons_d, bface_d, shape, dx, stream)
        # the first call may load the library's device code lazily; after
        # it, a call must leave the device's free memory unchanged
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        again = W.w5ct_conserved_totals_noalloc(cons_d, bface_d, shape, dx, stream)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert np.array_equal(again, got)        # fixed summation order
        absint = np.array([np.abs(cons[f]).sum() for f in range(5)] + [np.abs(bface[f]).sum() for f in range(3)])
        absint *= dx[0] * dx[1] * dx[2]
        assert np.all(np.abs(got - ref) <= 1e-13 * absint), (seed, got - ref)
    s.close()


def test_noalloc_rejects_grids_beyond_the_fixed_scratch(env):
    torch, I, W = env
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(W.W5ctError) as e:
        W.w5ct_conserved_totals_noalloc(dummy, dummy, (1024, 1024, 129), (1.0, 1.0, 1.0))
    assert e.value.code == W.W5CT_ERR_ARG
    assert "exceed" in W.w5ct_last_error(None)
