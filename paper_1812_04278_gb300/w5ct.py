"""ctypes binding of libw5ct (``include/w5ct.h``).

Every C entry point is exposed under its own name with argument
marshalling only; all arithmetic runs in the library's CUDA kernels.  A
non-zero return code raises :class:`W5ctError` carrying the library's error
text.  Device buffers passed with ``on_device=1`` are torch CUDA tensors
(or raw device addresses); host buffers are numpy float64 arrays.

Importing this module loads ``libw5ct.so`` from the package directory and
raises ImportError if it has not been built (``__graft_entry__.build()``):
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_longlong, c_void_p

import numpy as np

# W5CT_LIB may name an alternative build of the same library (same ABI)
_LIB_PATH = os.environ.get("W5CT_LIB") or os.path.join(os.path.dirname(os.path.abspath(__file__)), "libw5ct.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is missing: build it with __graft_entry__.build()")
_lib = ctypes.CDLL(_LIB_PATH)

W5CT_OK = 0
W5CT_ERR_ARG = -1
W5CT_ERR_CUDA = -2
W5CT_ERR_STATE = -3
W5CT_ERR_NONPHYSICAL = -4
W5CT_ERR_UNSUPPORTED = -5
W5CT_ERR_TIMEOUT = -6
W5CT_WENO_JS = 0
W5CT_WENO_Z = 1
W5CT_FP64 = 0
W5CT_FP32_BULK = 1
W5CT_FP64_DW = 2

EXPORTED = [
    "w5ct_config_default", "w5ct_create", "w5ct_destroy", "w5ct_set_stream", "w5ct_init_grid",
    "w5ct_set_state", "w5ct_get_state", "w5ct_step", "w5ct_step_dev", "w5ct_step_cfl",
    "w5ct_max_signal_speed", "w5ct_cfl_dt", "w5ct_div_b_norm", "w5ct_conserved_totals",
    "w5ct_status", "w5ct_synchronize", "w5ct_set_timing", "w5ct_sweep_timing",
    "w5ct_launch_count", "w5ct_last_error", "w5ct_conserved_totals_noalloc", "w5ct_step_graph",
    "w5ct_autotune", "w5ct_tile_variant", "w5ct_adjoint_step", "w5ct_misfit", "w5ct_ic_from_potential",
    "w5ct_ic_from_potential_adjoint", "w5ct_set_sweep_schedule", "w5ct_sweep_schedule",
    "w5ct_fused_wait_check",
]
W5CT_TUNE_MEASURE = -1
W5CT_TUNE_MODEL = -2
W5CT_NOALLOC_MAX_CELLS = 134217728


class w5ct_config(ctypes.Structure):
    _fields_ = [("gamma", c_double), ("cfl", c_double), ("weno_variant", c_int), ("precision", c_int),
                ("eps_js", c_double), ("eps_z", c_double), ("eps_b", c_double), ("floors", c_int),
                ("rho_min", c_double), ("p_min", c_double), ("stream", c_void_p)]


_DP = POINTER(c_double)
_VP = c_void_p
_sig = {
    "w5ct_config_default": [POINTER(w5ct_config)],
    "w5ct_create": [POINTER(w5ct_config), POINTER(c_void_p)],
    "w5ct_destroy": [_VP],
    "w5ct_set_stream": [_VP, _VP],
    "w5ct_init_grid": [_VP, c_int, POINTER(c_int), _DP],
    "w5ct_set_state": [_VP, c_int, _VP, _VP, c_int],
    "w5ct_get_state": [_VP, c_int, _VP, _VP, _VP, c_int],
    "w5ct_step": [_VP, c_double],
    "w5ct_step_dev": [_VP, _VP],
    "w5ct_step_cfl": [_VP, _VP],
    "w5ct_step_graph": [_VP, c_int],
    "w5ct_autotune": [_VP, c_int, c_int],
    "w5ct_tile_variant": [_VP, c_int, c_int, POINTER(c_int)],
    "w5ct_adjoint_step": [_VP, c_double, _VP, _VP, _VP, _VP],
    "w5ct_set_sweep_schedule": [_VP, c_int],
    "w5ct_sweep_schedule": [_VP, POINTER(c_int)],
    "w5ct_fused_wait_check": [_VP, c_longlong, POINTER(c_int)],
    "w5ct_misfit": [_VP, _VP, _VP, _DP, _VP, _VP],
    "w5ct_ic_from_potential": [POINTER(c_int), _DP, c_double, _DP, _VP, _VP, _VP, _VP, _VP, _VP, _VP],
    "w5ct_ic_from_potential_adjoint": [POINTER(c_int), _DP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP],
    "w5ct_max_signal_speed": [_VP, c_int, _DP],
    "w5ct_cfl_dt": [_VP, _DP],
    "w5ct_div_b_norm": [_VP, c_int, _DP, _DP],
    "w5ct_conserved_totals": [_VP, c_int, _DP],
    "w5ct_status": [_VP, POINTER(c_longlong), POINTER(c_int)],
    "w5ct_synchronize": [_VP],
    "w5ct_set_timing": [_VP, c_int],
    "w5ct_sweep_timing": [_VP, POINTER(c_longlong), _DP],
    "w5ct_launch_count": [_VP, POINTER(c_longlong)],
    "w5ct_conserved_totals_noalloc": [_VP, _VP, c_int, c_int, c_int, c_double, c_double, c_double, _DP, _VP],
}
for _name, _args in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = c_int
_lib.w5ct_last_error.argtypes = [_VP]
_lib.w5ct_last_error.restype = c_char_p


class W5ctError(RuntimeError):
    def __init__(self, code: int, where: str, text: str):
        super().__init__(f"{where} returned {code}: {text}")
        self.code = code


def w5ct_last_error(ctx=None) -> str:
    return _lib.w5ct_last_error(ctx).decode(errors="replace")


def _check(rc: int, where: str, ctx=None):
    if rc != 0:
        raise W5ctError(rc, where, w5ct_last_error(ctx))


def _addr(buf):
    """Address of a torch tensor, numpy array or integer; None -> NULL."""
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    if isinstance(buf, np.ndarray):
        assert buf.dtype == np.float64 and buf.flags.c_contiguous
        return buf.ctypes.data
    # torch tensor
    assert buf.is_contiguous() and str(buf.dtype) == "torch.float64"
    return buf.data_ptr()


# ------------------------------------------------------------------ entry points


def w5ct_config_default() -> w5ct_config:
    cfg = w5ct_config()
    _check(_lib.w5ct_config_default(ctypes.byref(cfg)), "w5ct_config_default")
    return cfg


def w5ct_create(cfg: w5ct_config):
    h = c_void_p()
    _check(_lib.w5ct_create(ctypes.byref(cfg), ctypes.byref(h)), "w5ct_create")
    return h


def w5ct_destroy(ctx):
    _check(_lib.w5ct_destroy(ctx), "w5ct_destroy")


def w5ct_set_stream(ctx, stream: int):
    _check(_lib.w5ct_set_stream(ctx, stream), "w5ct_set_stream", ctx)


def w5ct_init_grid(ctx, n3, dx3, npatch: int | None = None):
    """n3, dx3: one (nx, ny, nz) / (dx, dy, dz) triple, or npatch of them
    (nested or flattened); npatch defaults to the number of triples."""
    nf = [int(v) for v in np.asarray(n3).reshape(-1)]
    df = [float(v) for v in np.asarray(dx3, dtype=np.float64).reshape(-1)]
    if npatch is None:
        npatch = len(nf) // 3
    if len(nf) != 3 * max(npatch, 1) or len(df) != 3 * max(npatch, 1):
        raise ValueError(f"w5ct_init_grid: {npatch} patches need 3 sizes and 3 spacings each")
    n = (c_int * len(nf))(*nf)
    d = (c_double * len(df))(*df)
    _check(_lib.w5ct_init_grid(ctx, npatch, n, d), "w5ct_init_grid", ctx)


def w5ct_set_state(ctx, cons, bface, on_device: int, patch: int = 0):
    _check(_lib.w5ct_set_state(ctx, patch, _addr(cons), _addr(bface), on_device), "w5ct_set_state", ctx)


def w5ct_get_state(ctx, cons, bface, bcell, on_device: int, patch: int = 0):
    _check(_lib.w5ct_get_state(ctx, patch, _addr(cons), _addr(bface), _addr(bcell), on_device),
           "w5ct_get_state", ctx)


def w5ct_step(ctx, dt: float):
    _check(_lib.w5ct_step(ctx, float(dt)), "w5ct_step", ctx)


def w5ct_step_dev(ctx, dt_dev):
    _check(_lib.w5ct_step_dev(ctx, _addr(dt_dev)), "w5ct_step_dev", ctx)


def w5ct_step_cfl(ctx, dt_dev_out=None):
    _check(_lib.w5ct_step_cfl(ctx, _addr(dt_dev_out)), "w5ct_step_cfl", ctx)


def w5ct_step_graph(ctx, nsteps: int):
    _check(_lib.w5ct_step_graph(ctx, int(nsteps)), "w5ct_step_graph", ctx)


def w5ct_autotune(ctx, mode: int = W5CT_TUNE_MEASURE, reps: int = 3):
    _check(_lib.w5ct_autotune(ctx, int(mode), int(reps)), "w5ct_autotune", ctx)


def w5ct_set_sweep_schedule(ctx, schedule: int):
    _check(_lib.w5ct_set_sweep_schedule(ctx, int(schedule)), "w5ct_set_sweep_schedule", ctx)


def w5ct_sweep_schedule(ctx) -> int:
    out = c_int()
    _check(_lib.w5ct_sweep_schedule(ctx, ctypes.byref(out)), "w5ct_sweep_schedule", ctx)
    return out.value


def w5ct_fused_wait_check(ctx, spin_limit: int) -> int:
    """Status a synchronising call reports after a fused-step wait bounded by
    spin_limit sleeps expires (W5CT_ERR_TIMEOUT when the bound works)."""
    out = c_int()
    _check(_lib.w5ct_fused_wait_check(ctx, int(spin_limit), ctypes.byref(out)), "w5ct_fused_wait_check", ctx)
    return out.value


def w5ct_tile_variant(ctx, axis: int, patch: int):
    """(variant, BX, T2) of the tiles sweeping `patch` along `axis`."""
    out = (c_int * 3)()
    _check(_lib.w5ct_tile_variant(ctx, int(axis), int(patch), out), "w5ct_tile_variant", ctx)
    return tuple(out[:])


def w5ct_adjoint_step(ctx, dt: float, lam_q, lam_b, lam_q_out, lam_b_out):
    _check(_lib.w5ct_adjoint_step(ctx, float(dt), _addr(lam_q), _addr(lam_b), _addr(lam_q_out), _addr(lam_b_out)),
           "w5ct_adjoint_step", ctx)


def w5ct_misfit(ctx, target_cons, target_bface, lam_q, lam_b) -> float:
    out = c_double()
    _check(_lib.w5ct_misfit(ctx, _addr(target_cons), _addr(target_bface), ctypes.byref(out), _addr(lam_q),
                            _addr(lam_b)), "w5ct_misfit", ctx)
    return out.value


def _n3(shape):
    return (c_int * 3)(*[int(v) for v in shape])


def _d3(vals):
    return (c_double * 3)(*[float(v) for v in vals])


def w5ct_ic_from_potential(shape, dx, gamma, B0, rho, v, P, A, cons, bface, stream=None):
    _check(_lib.w5ct_ic_from_potential(_n3(shape), _d3(dx), float(gamma), _d3(B0), _addr(rho), _addr(v), _addr(P),
                                       _addr(A), _addr(cons), _addr(bface), stream), "w5ct_ic_from_potential")


def w5ct_ic_from_potential_adjoint(shape, dx, rho, v, bface, lam_cons, lam_bface, lam_rho, lam_v, lam_A, lam_b,
                                   stream=None):
    _check(_lib.w5ct_ic_from_potential_adjoint(_n3(shape), _d3(dx), _addr(rho), _addr(v), _addr(bface),
                                               _addr(lam_cons), _addr(lam_bface), _addr(lam_rho), _addr(lam_v),
                                               _addr(lam_A), _addr(lam_b), stream),
           "w5ct_ic_from_potential_adjoint")


def w5ct_max_signal_speed(ctx, patch: int = 0) -> np.ndarray:
    out = (c_double * 3)()
    _check(_lib.w5ct_max_signal_speed(ctx, patch, out), "w5ct_max_signal_speed", ctx)
    return np.array(out[:])


def w5ct_cfl_dt(ctx) -> float:
    out = c_double()
    _check(_lib.w5ct_cfl_dt(ctx, ctypes.byref(out)), "w5ct_cfl_dt", ctx)
    return out.value


def w5ct_div_b_norm(ctx, patch: int = 0):
    a, b = c_double(), c_double()
    _check(_lib.w5ct_div_b_norm(ctx, patch, ctypes.byref(a), ctypes.byref(b)), "w5ct_div_b_norm", ctx)
    return a.value, b.value


def w5ct_conserved_totals(ctx, patch: int = 0) -> np.ndarray:
    out = (c_double * 8)()
    _check(_lib.w5ct_conserved_totals(ctx, patch, out), "w5ct_conserved_totals", ctx)
    return np.array(out[:])


def w5ct_status(ctx):
    h, f = c_longlong(), c_int()
    _check(_lib.w5ct_status(ctx, ctypes.byref(h), ctypes.byref(f)), "w5ct_status", ctx)
    return h.value, f.value


def w5ct_synchronize(ctx):
    _check(_lib.w5ct_synchronize(ctx), "w5ct_synchronize", ctx)


def w5ct_set_timing(ctx, enable: bool):
    _check(_lib.w5ct_set_timing(ctx, int(bool(enable))), "w5ct_set_timing", ctx)


def w5ct_sweep_timing(ctx):
    n, ms = c_longlong(), c_double()
    _check(_lib.w5ct_sweep_timing(ctx, ctypes.byref(n), ctypes.byref(ms)), "w5ct_sweep_timing", ctx)
    return n.value, ms.value


def w5ct_launch_count(ctx) -> int:
    n = c_longlong()
    _check(_lib.w5ct_launch_count(ctx, ctypes.byref(n)), "w5ct_launch_count", ctx)
    return n.value


def w5ct_conserved_totals_noalloc(cons_dev, bface_dev, n3, dx3, stream=None) -> np.ndarray:
    """Totals of caller-owned device arrays without any device allocation
    (see include/w5ct.h); cons_dev / bface_dev are device buffers."""
    out = (c_double * 8)()
    _check(_lib.w5ct_conserved_totals_noalloc(_addr(cons_dev), _addr(bface_dev), int(n3[0]), int(n3[1]), int(n3[2]),
                                               float(dx3[0]), float(dx3[1]), float(dx3[2]), out, stream),
           "w5ct_conserved_totals_noalloc")
    return np.array(out[:])


# ------------------------------------------------------------------ convenience


def make_config(precision=W5CT_FP64, weno_variant=W5CT_WENO_Z, gamma=5.0 / 3.0, cfl=0.8, floors=0,
                rho_min=1e-8, p_min=1e-8, stream=None, eps_js=1e-6, eps_z=1e-40, eps_b=1e-30) -> w5ct_config:
    cfg = w5ct_config_default()
    cfg.precision = precision
    cfg.weno_variant = weno_variant
    cfg.gamma = gamma
    cfg.cfl = cfl
    cfg.floors = floors
    cfg.rho_min = rho_min
    cfg.p_min = p_min
    cfg.eps_js = eps_js
    cfg.eps_z = eps_z
    cfg.eps_b = eps_b
    cfg.stream = stream
    return cfg


class Solver:
    """One periodic patch on the GPU: owns a context and forwards to the C ABI."""

    def __init__(self, shape, dx, cfg: w5ct_config | None = None, stream: int | None = None):
        cfg = cfg if cfg is not None else make_config()
        if stream is not None:
            cfg.stream = stream
        self.cfg = cfg
        self.ctx = w5ct_create(cfg)
        self.shape = tuple(int(s) for s in shape)
        self.dx = tuple(float(d) for d in (dx if not np.isscalar(dx) else (dx, dx, dx)))
        self.n = self.shape[0] * self.shape[1] * self.shape[2]
        w5ct_init_grid(self.ctx, self.shape, self.dx)

    def close(self):
        if self.ctx:
            w5ct_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, cons, bface):
        if isinstance(cons, np.ndarray):
            cons = np.ascontiguousarray(cons, dtype=np.float64)
            bface = np.ascontiguousarray(bface, dtype=np.float64)
            assert cons.size == 5 * self.n and bface.size == 3 * self.n
            w5ct_set_state(self.ctx, cons, bface, 0)
        else:
            assert cons.is_cuda and cons.numel() == 5 * self.n and bface.numel() == 3 * self.n
            w5ct_set_state(self.ctx, cons.contiguous(), bface.contiguous(), 1)

    def get_state(self):
        nx, ny, nz = self.shape
        cons = np.empty((5, nz, ny, nx))
        bface = np.empty((3, nz, ny, nx))
        bcell = np.empty((3, nz, ny, nx))
        w5ct_get_state(self.ctx, cons, bface, bcell, 0)
        return cons, bface, bcell

    def step(self, dt: float):
        w5ct_step(self.ctx, dt)

    def step_cfl(self, dt_dev_out=None):
        w5ct_step_cfl(self.ctx, dt_dev_out)

    def max_signal_speed(self):
        return w5ct_max_signal_speed(self.ctx)

    def cfl_dt(self):
        return w5ct_cfl_dt(self.ctx)

    def div_b_norm(self):
        return w5ct_div_b_norm(self.ctx)

    def conserved_totals(self):
        return w5ct_conserved_totals(self.ctx)

    def status(self):
        return w5ct_status(self.ctx)

    def synchronize(self):
        w5ct_synchronize(self.ctx)


class Batch:
    """Several independent periodic patches advanced together by one context
    (every launch covers the tiles of all patches; w5ct_step_graph replays a
    captured step)."""

    def __init__(self, shapes, dxs, cfg: w5ct_config | None = None, stream: int | None = None):
        cfg = cfg if cfg is not None else make_config()
        if stream is not None:
            cfg.stream = stream
        self.cfg = cfg
        self.ctx = w5ct_create(cfg)
        self.shapes = [tuple(int(s) for s in sh) for sh in shapes]
        self.dxs = [tuple(float(d) for d in dx) for dx in dxs]
        self.npatch = len(self.shapes)
        w5ct_init_grid(self.ctx, self.shapes, self.dxs, npatch=self.npatch)

    def close(self):
        if self.ctx:
            w5ct_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, p, cons, bface):
        if isinstance(cons, np.ndarray):
            w5ct_set_state(self.ctx, np.ascontiguousarray(cons, dtype=np.float64),
                           np.ascontiguousarray(bface, dtype=np.float64), 0, patch=p)
        else:
            w5ct_set_state(self.ctx, cons.contiguous(), bface.contiguous(), 1, patch=p)

    def get_state(self, p):
        nx, ny, nz = self.shapes[p]
        cons = np.empty((5, nz, ny, nx))
        bface = np.empty((3, nz, ny, nx))
        bcell = np.empty((3, nz, ny, nx))
        w5ct_get_state(self.ctx, cons, bface, bcell, 0, patch=p)
        return cons, bface, bcell

    def step(self, dt):
        w5ct_step(self.ctx, dt)

    def step_dev(self, dts_dev):
        """One step, patch p taking dts_dev[p] (device buffer of npatch doubles)."""
        w5ct_step_dev(self.ctx, dts_dev)

    def step_cfl(self, dt_dev_out=None):
        w5ct_step_cfl(self.ctx, dt_dev_out)

    def step_graph(self, nsteps):
        w5ct_step_graph(self.ctx, nsteps)

    def autotune(self, mode=W5CT_TUNE_MEASURE, reps=3):
        w5ct_autotune(self.ctx, mode, reps)

    def set_schedule(self, schedule):
        w5ct_set_sweep_schedule(self.ctx, schedule)

    def schedule(self):
        return w5ct_sweep_schedule(self.ctx)

    def tile_variants(self):
        """Number of patches per (axis, variant)."""
        out = np.zeros((3, 4), dtype=np.int64)
        for a in range(3):
            for p in range(self.npatch):
                out[a, w5ct_tile_variant(self.ctx, a, p)[0]] += 1
        return out

    def max_signal_speed(self, p):
        return w5ct_max_signal_speed(self.ctx, p)

    def div_b_norm(self, p):
        return w5ct_div_b_norm(self.ctx, p)

    def conserved_totals(self, p):
        return w5ct_conserved_totals(self.ctx, p)

    def status(self):
        return w5ct_status(self.ctx)

    def synchronize(self):
        w5ct_synchronize(self.ctx)
