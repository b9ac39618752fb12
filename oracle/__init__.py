"""ctypes wrapper of the plain FP64 CPU oracle (``w5ct_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, obviously-correct CPU
implementation of the WENO5 + constrained-transport MHD step of Donnert et
al. (arXiv:1812.04278) that the CUDA library is checked against.  Only the
test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.

Functions whose correctness is pinned only indirectly (through the
integration tests rather than a closed form) are marked in their docstrings.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from ctypes import POINTER, c_double, c_int, c_long, c_longlong, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "w5ct_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

WENO_JS, WENO_Z, WENO_Z_PRINTED = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (IEEE double, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class OracleConfig(ctypes.Structure):
    _fields_ = [("gamma", c_double), ("cfl", c_double), ("weno_variant", c_int),
                ("eps_js", c_double), ("eps_z", c_double), ("eps_b", c_double),
                ("floors", c_int), ("rho_min", c_double), ("p_min", c_double)]


def make_config(gamma=5.0 / 3.0, cfl=0.8, weno_variant=WENO_Z, eps_js=1e-6, eps_z=1e-40,
                eps_b=1e-30, floors=0, rho_min=1e-8, p_min=1e-8) -> OracleConfig:
    return OracleConfig(gamma, cfl, weno_variant, eps_js, eps_z, eps_b, floors, rho_min, p_min)


_lib = None
_DP = POINTER(c_double)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp = c_void_p
        lib.ora_create.argtypes = [POINTER(OracleConfig), POINTER(vp)]
        lib.ora_destroy.argtypes = [vp]
        lib.ora_init_grid.argtypes = [vp, c_int, c_int, c_int, c_double, c_double, c_double]
        lib.ora_set_state.argtypes = [vp, _DP, _DP]
        lib.ora_get_state.argtypes = [vp, _DP, _DP, _DP]
        lib.ora_step.argtypes = [vp, c_double]
        lib.ora_step_linear.argtypes = [vp, c_double, _DP]
        lib.ora_max_signal_speed.argtypes = [vp, _DP]
        lib.ora_cfl_dt.argtypes = [vp, _DP]
        lib.ora_div_b_norm.argtypes = [vp, _DP, _DP]
        lib.ora_conserved_totals.argtypes = [vp, _DP]
        lib.ora_status.argtypes = [vp, POINTER(c_longlong), POINTER(c_int)]
        lib.ora1d_step.argtypes = [POINTER(OracleConfig), c_int, c_double, c_double, _DP, c_double]
        lib.ora_eigensystem.argtypes = [_DP, c_double, c_double, _DP, _DP, _DP]
        lib.ora_eigensystem.restype = None
        lib.ora_frame_flux.argtypes = [_DP, c_double, _DP]
        lib.ora_frame_flux.restype = None
        lib.ora_wave_speeds.argtypes = [c_double, _DP, _DP]
        lib.ora_wave_speeds.restype = None
        lib.ora_phi_n.argtypes = [c_double, c_double, c_double, c_double, POINTER(OracleConfig)]
        lib.ora_phi_n.restype = c_double
        lib.ora_weno_char_flux.argtypes = [_DP, _DP, c_double, POINTER(OracleConfig)]
        lib.ora_weno_char_flux.restype = c_double
        lib.ora_num_threads.restype = c_int
        lib.ora_set_num_threads.argtypes = [c_int]
        lib.ora_set_num_threads.restype = c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"oracle {what} returned {rc}")


def num_threads() -> int:
    return int(_load().ora_num_threads())


def set_num_threads(n: int) -> None:
    """Host threads of the oracle's following calls."""
    _check(_load().ora_set_num_threads(int(n)), "set_num_threads")


class Oracle:
    """One periodic patch advanced by the oracle (mirrors the C-ABI calls)."""

    def __init__(self, shape, dx, cfg: OracleConfig | None = None):
        self.lib = _load()
        self.cfg = cfg if cfg is not None else make_config()
        self.h = c_void_p()
        _check(self.lib.ora_create(ctypes.byref(self.cfg), ctypes.byref(self.h)), "create")
        nx, ny, nz = (int(s) for s in shape)
        if np.isscalar(dx):
            dx = (dx, dx, dx)
        self.shape = (nx, ny, nz)
        self.dx = tuple(float(d) for d in dx)
        self.n = nx * ny * nz
        _check(self.lib.ora_init_grid(self.h, nx, ny, nz, *self.dx), "init_grid")

    def close(self):
        if self.h:
            self.lib.ora_destroy(self.h)
            self.h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # arrays are (nf, nz, ny, nx) float64, x fastest
    def set_state(self, cons: np.ndarray, bface: np.ndarray):
        cons = np.ascontiguousarray(cons, dtype=np.float64)
        bface = np.ascontiguousarray(bface, dtype=np.float64)
        assert cons.size == 5 * self.n and bface.size == 3 * self.n
        _check(self.lib.ora_set_state(self.h, _ptr(cons), _ptr(bface)), "set_state")

    def get_state(self):
        nx, ny, nz = self.shape
        cons = np.empty((5, nz, ny, nx))
        bface = np.empty((3, nz, ny, nx))
        bcell = np.empty((3, nz, ny, nx))
        _check(self.lib.ora_get_state(self.h, _ptr(cons), _ptr(bface), _ptr(bcell)), "get_state")
        return cons, bface, bcell

    def step(self, dt: float):
        _check(self.lib.ora_step(self.h, float(dt)), "step")

    def step_linear(self, dt: float, M):
        m = np.ascontiguousarray(np.asarray(M, dtype=np.float64).reshape(4))
        _check(self.lib.ora_step_linear(self.h, float(dt), _ptr(m)), "step_linear")

    def max_signal_speed(self) -> np.ndarray:
        out = np.zeros(3)
        _check(self.lib.ora_max_signal_speed(self.h, _ptr(out)), "max_signal_speed")
        return out

    def cfl_dt(self) -> float:
        out = np.zeros(1)
        _check(self.lib.ora_cfl_dt(self.h, _ptr(out)), "cfl_dt")
        return float(out[0])

    def div_b_norm(self):
        a, b = np.zeros(1), np.zeros(1)
        _check(self.lib.ora_div_b_norm(self.h, _ptr(a), _ptr(b)), "div_b_norm")
        return float(a[0]), float(b[0])

    def conserved_totals(self) -> np.ndarray:
        out = np.zeros(8)
        _check(self.lib.ora_conserved_totals(self.h, _ptr(out)), "conserved_totals")
        return out

    def status(self):
        hits, bad = c_longlong(), c_int()
        _check(self.lib.ora_status(self.h, ctypes.byref(hits), ctypes.byref(bad)), "status")
        return int(hits.value), int(bad.value)


def step1d(u: np.ndarray, dx: float, Bx: float, dt: float, cfg: OracleConfig | None = None) -> np.ndarray:
    """One RK4 step of the 1-D program (Sec. 3.1.1) on u = (7, nx):
    (rho, m_x, m_y, m_z, B_y, B_z, E).  Returns the new array."""
    lib = _load()
    cfg = cfg if cfg is not None else make_config()
    a = np.ascontiguousarray(u, dtype=np.float64).copy()
    assert a.shape[0] == 7
    _check(lib.ora1d_step(ctypes.byref(cfg), a.shape[1], float(dx), float(Bx), _ptr(a), float(dt)), "1d step")
    return a


def eigensystem(w, gamma=5.0 / 3.0, eps_b=1e-30):
    """Appendix A at primitive state w = (rho, v_n, v_t1, v_t2, B_n, B_t1, B_t2, P).
    Returns (L, R, lam); row m of L / R is the m-th left / right eigenvector."""
    lib = _load()
    w = np.ascontiguousarray(w, dtype=np.float64)
    L, R, lam = np.zeros(49), np.zeros(49), np.zeros(7)
    lib.ora_eigensystem(_ptr(w), gamma, eps_b, _ptr(L), _ptr(R), _ptr(lam))
    return L.reshape(7, 7), R.reshape(7, 7), lam


def frame_flux(w, E):
    lib = _load()
    w = np.ascontiguousarray(w, dtype=np.float64)
    F = np.zeros(7)
    lib.ora_frame_flux(_ptr(w), float(E), _ptr(F))
    return F


def wave_speeds(w, gamma=5.0 / 3.0):
    """(c_s, c_A, c_slow, c_f) at primitive state w."""
    lib = _load()
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros(4)
    lib.ora_wave_speeds(gamma, _ptr(w), _ptr(out))
    return out


def phi_n(a, b, c, d, cfg: OracleConfig | None = None) -> float:
    cfg = cfg if cfg is not None else make_config()
    return float(_load().ora_phi_n(a, b, c, d, ctypes.byref(cfg)))


def weno_char_flux(Fs, qs, alpha, cfg: OracleConfig | None = None) -> float:
    cfg = cfg if cfg is not None else make_config()
    Fs = np.ascontiguousarray(Fs, dtype=np.float64)
    qs = np.ascontiguousarray(qs, dtype=np.float64)
    return float(_load().ora_weno_char_flux(_ptr(Fs), _ptr(qs), float(alpha), ctypes.byref(cfg)))
