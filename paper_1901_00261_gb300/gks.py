"""Python binding of the C ABI in include/gks.h (argument marshalling only).

Every step of the scheme runs in the CUDA kernels of libgks_gb300.so; this module only
loads the library, converts arguments and raises on error codes.  There is no CPU
fallback: if the library cannot be built or loaded, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

GKS_OK, GKS_EINVAL, GKS_ECUDA, GKS_ENOMEM, GKS_ENONPHYSICAL, GKS_ETIMEOUT = 0, -1, -2, -3, -4, -5
RECON_LINEAR, RECON_WENOZ = 0, 1
PREC_FP64, PREC_FP32_BULK = 0, 1
BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECTING, BC_ISOTHERMAL = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


class GksError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"gks error {code}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
                ("precision", ctypes.c_int),
                ("weno_eps", ctypes.c_double),
                ("eps_tau", ctypes.c_double), ("C_tau", ctypes.c_double),
                ("use_graph", ctypes.c_int),
                ("tau_mode", ctypes.c_int),
                ("stream", ctypes.c_void_p),
                ("tan_mode", ctypes.c_int),
                ("wall_T", ctypes.c_double * 4), ("wall_u", ctypes.c_double * 4),
                ("coef_mode", ctypes.c_int)]


# Every symbol include/gks.h declares, with (restype, argtypes).
_DP = ctypes.POINTER(ctypes.c_double)
_DPP = ctypes.POINTER(ctypes.POINTER(ctypes.c_double))
SIGNATURES = {
    "gks_default_opts": (None, [ctypes.POINTER(Opts)]),
    "gks_create": (ctypes.c_void_p, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Opts)]),
    "gks_last_error": (ctypes.c_char_p, []),
    "gks_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gks_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gks_set_state_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gks_get_state_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gks_get_rows_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "gks_set_rows_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "gks_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "gks_steps": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int]),
    "gks_max_wavespeed": (ctypes.c_int, [ctypes.c_void_p, _DP]),
    "gks_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "gks_step_host_async": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 6 + [ctypes.c_double]),
    "gks_state_device_ptrs": (ctypes.c_int, [ctypes.c_void_p, _DPP, _DPP, _DPP]),
    "gks_launches_per_step": (ctypes.c_int, [ctypes.c_void_p]),
    "gks_destroy": (None, [ctypes.c_void_p]),
    "gks_steps_timed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, _DP]),
    "gks_probe_alu_peak": (ctypes.c_int, [ctypes.c_int, _DP]),
    "gks_probe_time_coefs": (ctypes.c_int, [_DP, ctypes.c_int, ctypes.c_double, _DP]),
    "gks_probe_time_coefs_single": (ctypes.c_int, [_DP, ctypes.c_int, ctypes.c_double, _DP]),
    "gks_probe_rcp64": (ctypes.c_int, [_DP, ctypes.c_int, _DP]),
    "gks_probe_d2f": (ctypes.c_int, [_DP, ctypes.c_int, ctypes.c_void_p]),
    "gks_step_1d_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_void_p]),
    "gks_static_last_error": (ctypes.c_char_p, []),
}
STATIC_MAX_NX = 16384


class Problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("order", ctypes.c_int), ("recon", ctypes.c_int),
                ("gamma", ctypes.c_double), ("mu", ctypes.c_double), ("Pr", ctypes.c_double),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int)]


_VP = ctypes.c_void_p
SIGNATURES.update({
    "gks_batch_create": (_VP, [ctypes.c_int, ctypes.POINTER(Problem), _VP]),
    "gks_batch_last_error": (ctypes.c_char_p, []),
    "gks_batch_set_state": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP]),
    "gks_batch_get_state": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP]),
    "gks_batch_steps": (ctypes.c_int, [_VP, _DP, ctypes.c_int]),
    "gks_batch_step": (ctypes.c_int, [_VP, _DP]),
    "gks_batch_max_wavespeed": (ctypes.c_int, [_VP, _DP]),
    "gks_batch_sync": (ctypes.c_int, [_VP]),
    "gks_batch_config": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "gks_batch_set_config": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int]),
    "gks_batch_autotune": (ctypes.c_int, [_VP, _DP, ctypes.c_int, ctypes.c_char_p, ctypes.c_int]),
    "gks_batch_destroy": (None, [_VP]),
    "gks_batch_reset": (ctypes.c_int, [_VP]),
    "gks_batch_problem_status": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int)]),
    "gks_batch_debug_missing_producer": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_double]),
})


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libgks_gb300.so (building it first if needed).  Raises if it cannot."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libgks_gb300.so not found at {path}")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def last_error() -> str:
    return lib().gks_last_error().decode(errors="replace")


def _check(rc: int):
    if rc != GKS_OK:
        raise GksError(rc, last_error())


def default_opts() -> Opts:
    o = Opts()
    lib().gks_default_opts(ctypes.byref(o))
    return o


def _host_ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return ctypes.c_void_p(a.ctypes.data)


class Solver:
    """A gks_ctx: the two-stage compact GKS on an nx x ny grid (ny == 1: 1D).

    Host state arrays are float64 [nvar][ny][nx].  ``stream`` is a CUDA stream handle
    (e.g. ``torch.cuda.current_stream().cuda_stream``) or None."""

    def __init__(self, nx: int, ny: int = 1, gamma: float = 1.4, mu: float = 0.0, Pr: float = 1.0,
                 order: int = 6, recon: int = RECON_LINEAR, x0: float = 0.0, x1: float = 1.0,
                 y0: float = 0.0, y1: float = 1.0, bc_x: int = BC_PERIODIC, bc_y: int = BC_PERIODIC,
                 weno_eps: float = 1e-6, use_graph: bool = True, stream=None,
                 precision: int = PREC_FP64, tau_mode: int = 0, eps_tau: float = 0.01,
                 C_tau: float = 1.0, tan_mode: int = 0, wall_T=(1.0, 1.0, 1.0, 1.0),
                 wall_u=(0.0, 0.0, 0.0, 0.0), coef_mode: int = 0):
        L = lib()
        o = default_opts()
        o.precision = precision
        o.x0, o.x1, o.y0, o.y1 = x0, x1, y0, y1
        o.bc_x, o.bc_y = bc_x, bc_y
        o.weno_eps = weno_eps
        o.use_graph = 1 if use_graph else 0
        o.tau_mode = tau_mode
        o.tan_mode = tan_mode
        o.coef_mode = coef_mode
        for k in range(4):
            o.wall_T[k], o.wall_u[k] = float(wall_T[k]), float(wall_u[k])
        o.eps_tau, o.C_tau = eps_tau, C_tau
        o.stream = stream
        self._h = L.gks_create(nx, ny, gamma, mu, Pr, order, recon, ctypes.byref(o))
        if not self._h:
            raise GksError(GKS_EINVAL, last_error())
        self.nx, self.ny = nx, ny
        self.dim = 2 if ny > 1 else 1
        self.nv = self.dim + 2

    @classmethod
    def from_state(cls, st, **kw):
        """Solver configured from an inputs.State (grid, BCs, physics, order, recon)."""
        kw.setdefault("wall_T", st.wall_T)
        kw.setdefault("wall_u", st.wall_u)
        s = cls(st.nx, st.ny, st.gamma, st.mu, st.Pr, st.order, st.recon, st.x0, st.x1,
                st.y0, st.y1, st.bc_x, st.bc_y, **kw)
        s.set_state(st.W, st.Wx, st.Wy)
        return s

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib().gks_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.nv, self.ny, self.nx)

    def set_state(self, W, Wx, Wy=None):
        W = np.ascontiguousarray(W, dtype=np.float64).reshape(self.shape)
        Wx = np.ascontiguousarray(Wx, dtype=np.float64).reshape(self.shape)
        Wy = None if self.dim == 1 else np.ascontiguousarray(Wy, dtype=np.float64).reshape(self.shape)
        _check(lib().gks_set_state(self._h, _host_ptr(W), _host_ptr(Wx), _host_ptr(Wy)))

    def get_state(self):
        W = np.empty(self.shape)
        Wx = np.empty(self.shape)
        Wy = np.empty(self.shape) if self.dim == 2 else None
        _check(lib().gks_get_state(self._h, _host_ptr(W), _host_ptr(Wx), _host_ptr(Wy)))
        return W, Wx, Wy

    def set_state_device(self, W_ptr: int, Wx_ptr: int, Wy_ptr: int | None = None):
        _check(lib().gks_set_state_device(self._h, ctypes.c_void_p(W_ptr), ctypes.c_void_p(Wx_ptr),
                                          ctypes.c_void_p(Wy_ptr) if Wy_ptr else None))

    def get_state_device(self, W_ptr: int, Wx_ptr: int, Wy_ptr: int | None = None):
        _check(lib().gks_get_state_device(self._h, ctypes.c_void_p(W_ptr), ctypes.c_void_p(Wx_ptr),
                                          ctypes.c_void_p(Wy_ptr) if Wy_ptr else None))

    def get_rows_device(self, j0: int, nrows: int, buf_ptr: int):
        """Rows [j0, j0 + nrows) of W, Wx, Wy into the device buffer [3][nvar][nrows][nx]."""
        _check(lib().gks_get_rows_device(self._h, int(j0), int(nrows), ctypes.c_void_p(buf_ptr)))

    def set_rows_device(self, j0: int, nrows: int, buf_ptr: int):
        """Rows [j0, j0 + nrows) of W, Wx, Wy from the device buffer [3][nvar][nrows][nx]."""
        _check(lib().gks_set_rows_device(self._h, int(j0), int(nrows), ctypes.c_void_p(buf_ptr)))

    def step(self, dt: float):
        _check(lib().gks_step(self._h, float(dt)))

    def steps(self, dt: float, n: int):
        _check(lib().gks_steps(self._h, float(dt), int(n)))

    def max_wavespeed(self) -> float:
        v = ctypes.c_double()
        _check(lib().gks_max_wavespeed(self._h, ctypes.byref(v)))
        return v.value

    def step_host_async(self, ins, outs, dt: float):
        """Pipelined host-to-host step (gks_step_host_async): ins = (W, Wx[, Wy]) are copied
        in, advanced one step of dt, and written to outs = (W, Wx[, Wy]) (C-contiguous float64
        arrays of the state's shape, ideally pinned).  Returns at once; the arrays must stay
        alive, and outs unread, until sync()."""
        arrs = list(ins) + [None] * (3 - len(ins)) + list(outs) + [None] * (3 - len(outs))
        for a in arrs[:self.dim + 1] + arrs[3:4 + self.dim]:
            if a.shape != self.shape or a.dtype != np.float64 or not a.flags.c_contiguous:
                raise ValueError("state arrays must be C-contiguous float64 of shape %s" % (self.shape,))
        p = [_host_ptr(a) if k % 3 <= self.dim else None for k, a in enumerate(arrs)]
        _check(lib().gks_step_host_async(self._h, *p, float(dt)))

    def sync(self):
        _check(lib().gks_sync(self._h))

    def device_ptrs(self):
        a, b, c = ctypes.POINTER(ctypes.c_double)(), ctypes.POINTER(ctypes.c_double)(), ctypes.POINTER(ctypes.c_double)()
        _check(lib().gks_state_device_ptrs(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        addr = lambda p: ctypes.cast(p, ctypes.c_void_p).value
        return addr(a), addr(b), addr(c) if self.dim == 2 else None

    def launches_per_step(self) -> int:
        return int(lib().gks_launches_per_step(self._h))

    def steps_timed(self, dt: float, n: int) -> np.ndarray:
        """Run n steps with event-bracketed launches; returns summed ms per launch slot."""
        ms = np.zeros(self.launches_per_step())
        _check(lib().gks_steps_timed(self._h, float(dt), int(n),
                                     ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return ms


def probe_alu_peak(fp64: bool = True) -> float:
    """FLOP/s of an FMA-chain kernel over the whole device (roofline denominator)."""
    v = ctypes.c_double()
    _check(lib().gks_probe_alu_peak(1 if fp64 else 0, ctypes.byref(v)))
    return v.value


def probe_time_coefs(theta, dt: float, single: bool = False) -> np.ndarray:
    """The face kernels' FP64 time-integration coefficients (a0, a1, b0, b1) for each
    theta = tau/dt, evaluated on the device (gks_probe_time_coefs, or with single the
    single-precision form's truncation, gks_probe_time_coefs_single); shape (n, 4)."""
    th = np.ascontiguousarray(theta, dtype=np.float64).ravel()
    out = np.zeros((th.size, 4))
    fn = lib().gks_probe_time_coefs_single if single else lib().gks_probe_time_coefs
    _check(fn(th.ctypes.data_as(_DP), th.size, float(dt), out.ctypes.data_as(_DP)))
    return out


def probe_rcp64(x) -> np.ndarray:
    """The FP32-bulk sweeps' FP64 reciprocal of each x, evaluated on the device."""
    xx = np.ascontiguousarray(x, dtype=np.float64).ravel()
    out = np.zeros(xx.size)
    _check(lib().gks_probe_rcp64(xx.ctypes.data_as(_DP), xx.size, out.ctypes.data_as(_DP)))
    return out


def probe_d2f(x) -> np.ndarray:
    """The FP32-bulk form's double -> float rounding of each x, evaluated on the device."""
    xx = np.ascontiguousarray(x, dtype=np.float64).ravel()
    out = np.zeros(xx.size, dtype=np.float32)
    _check(lib().gks_probe_d2f(xx.ctypes.data_as(_DP), xx.size, ctypes.c_void_p(out.ctypes.data)))
    return out


def _bcheck(rc: int):
    if rc != GKS_OK:
        raise GksError(rc, lib().gks_batch_last_error().decode(errors="replace"))


class Batch:
    """Many independent problems advanced together (FP32-bulk form, persistent launch).

    ``states`` is a list of inputs.State (grid, domain, BCs, physics, order, recon)."""

    def __init__(self, states, stream=None):
        L = lib()
        arr = (Problem * len(states))()
        for k, st in enumerate(states):
            arr[k] = Problem(st.nx, st.ny, st.order, st.recon, st.gamma, st.mu, st.Pr,
                             st.x0, st.x1, st.y0, st.y1, st.bc_x, st.bc_y)
        self._h = L.gks_batch_create(len(states), arr, stream)
        if not self._h:
            raise GksError(GKS_EINVAL, L.gks_batch_last_error().decode(errors="replace"))
        self.shapes = [((2 if st.ny > 1 else 1) + 2, st.ny, st.nx) for st in states]
        self.n = len(states)
        for k, st in enumerate(states):
            self.set_state(k, st.W, st.Wx, st.Wy)

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib().gks_batch_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, i, W, Wx, Wy=None):
        shp = self.shapes[i]
        W = np.ascontiguousarray(W, dtype=np.float64).reshape(shp)
        Wx = np.ascontiguousarray(Wx, dtype=np.float64).reshape(shp)
        Wy = None if shp[1] == 1 else np.ascontiguousarray(Wy, dtype=np.float64).reshape(shp)
        _bcheck(lib().gks_batch_set_state(self._h, i, _host_ptr(W), _host_ptr(Wx), _host_ptr(Wy)))

    def get_state(self, i):
        shp = self.shapes[i]
        W, Wx = np.empty(shp), np.empty(shp)
        Wy = np.empty(shp) if shp[1] > 1 else None
        _bcheck(lib().gks_batch_get_state(self._h, i, _host_ptr(W), _host_ptr(Wx), _host_ptr(Wy)))
        return W, Wx, Wy

    def _dt(self, dt):
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (self.n,)))
        return a, a.ctypes.data_as(_DP)

    def steps(self, dt, n: int):
        a, p = self._dt(dt)
        _bcheck(lib().gks_batch_steps(self._h, p, int(n)))

    def max_wavespeed(self) -> np.ndarray:
        out = np.zeros(self.n)
        _bcheck(lib().gks_batch_max_wavespeed(self._h, out.ctypes.data_as(_DP)))
        return out

    def sync(self):
        _bcheck(lib().gks_batch_sync(self._h))

    def config(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        _bcheck(lib().gks_batch_config(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def set_config(self, faces_per_thread: int, blocks_per_sm: int):
        _bcheck(lib().gks_batch_set_config(self._h, faces_per_thread, blocks_per_sm))

    def problem_status(self):
        """Per-problem status: GKS_OK, or GKS_ENONPHYSICAL for a problem that met a non-physical
        state (frozen since)."""
        out = np.zeros(self.n, dtype=np.int32)
        _bcheck(lib().gks_batch_problem_status(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        return out

    def reset(self):
        _bcheck(lib().gks_batch_reset(self._h))

    def debug_missing_producer(self, problem: int, phase: int, wait_seconds: float):
        _bcheck(lib().gks_batch_debug_missing_producer(self._h, problem, phase, wait_seconds))

    def autotune(self, dt, steps: int = 3) -> str:
        a, p = self._dt(dt)
        buf = ctypes.create_string_buffer(4096)
        _bcheck(lib().gks_batch_autotune(self._h, p, int(steps), buf, 4096))
        return buf.value.decode()
