"""Host-side checks of the C ABI (no GPU needed): the library builds and
loads, exports every entry point declared in include/w5ct.h, and validates
its arguments before touching the device."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "w5ct.h")


@pytest.fixture(scope="module")
def w5():
    from paper_1812_04278_gb300 import build
    build.build()
    from paper_1812_04278_gb300 import w5ct
    return w5ct


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(w5ct_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("w5ct_create", "w5ct_init_grid", "w5ct_set_state", "w5ct_step", "w5ct_max_signal_speed",
                 "w5ct_div_b_norm", "w5ct_conserved_totals", "w5ct_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(w5):
    for name in declared_functions():
        assert hasattr(w5._lib, name), name
    assert set(declared_functions()) == set(w5.EXPORTED)


def test_config_defaults_are_the_papers(w5):
    cfg = w5.w5ct_config_default()
    assert cfg.gamma == 5.0 / 3.0 and cfg.cfl == 0.8
    assert cfg.eps_js == 1e-6 and cfg.eps_z == 1e-40 and cfg.eps_b == 1e-30
    assert cfg.floors == 0 and cfg.weno_variant == w5.W5CT_WENO_Z and cfg.precision == w5.W5CT_FP64


@pytest.mark.parametrize("field,value", [("gamma", 1.0), ("cfl", 0.0), ("weno_variant", 7), ("precision", 3),
                                         ("eps_js", 0.0), ("eps_b", -1.0)])
def test_create_rejects_bad_config(w5, field, value):
    cfg = w5.w5ct_config_default()
    setattr(cfg, field, value)
    with pytest.raises(w5.W5ctError) as e:
        w5.w5ct_create(cfg)
    assert e.value.code == w5.W5CT_ERR_ARG
    assert len(w5.w5ct_last_error(None)) > 0


@pytest.mark.parametrize("precision", ["W5CT_FP64", "W5CT_FP32_BULK", "W5CT_FP64_DW"])
def test_create_accepts_every_precision(w5, precision):
    cfg = w5.w5ct_config_default()
    cfg.precision = getattr(w5, precision)
    w5.w5ct_destroy(w5.w5ct_create(cfg))


def test_create_and_destroy_without_device_work(w5):
    ctx = w5.w5ct_create(w5.w5ct_config_default())
    with pytest.raises(w5.W5ctError) as e:
        w5.w5ct_step(ctx, 0.1)            # no grid yet: rejected on the host
    assert e.value.code == w5.W5CT_ERR_ARG or e.value.code == w5.W5CT_ERR_STATE
    with pytest.raises(w5.W5ctError) as e:
        w5.w5ct_init_grid(ctx, (8, 8, 8), (0.1, 0.1, 0.1), npatch=0)
    assert e.value.code == w5.W5CT_ERR_ARG
    with pytest.raises(w5.W5ctError) as e:
        w5.w5ct_init_grid(ctx, (0, 8, 8), (0.1, 0.1, 0.1))
    assert e.value.code == w5.W5CT_ERR_ARG
    with pytest.raises(w5.W5ctError) as e:      # second patch invalid
        w5.w5ct_init_grid(ctx, [(8, 8, 8), (4, -1, 4)], [(0.1, 0.1, 0.1)] * 2)
    assert e.value.code == w5.W5CT_ERR_ARG
    with pytest.raises(ValueError):             # buffers shorter than 3 x npatch
        w5.w5ct_init_grid(ctx, (8, 8, 8), (0.1, 0.1, 0.1), npatch=2)
    w5.w5ct_destroy(ctx)


def test_batched_entry_points_validate_on_the_host(w5):
    """The schedule setter, the fused-wait check and the adjoint entry points
    reject a context without a grid or state before any device work."""
    ctx = w5.w5ct_create(w5.w5ct_config_default())
    for call in (lambda: w5.w5ct_set_sweep_schedule(ctx, 2),
                 lambda: w5.w5ct_fused_wait_check(ctx, 1000),
                 lambda: w5.w5ct_tile_variant(ctx, 0, 0)):
        with pytest.raises(w5.W5ctError) as e:
            call()
        assert e.value.code in (w5.W5CT_ERR_ARG, w5.W5CT_ERR_STATE)
    w5.w5ct_destroy(ctx)
