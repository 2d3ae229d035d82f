"""Plain FP64 CPU oracle of the compact 6th/8th-order gas-kinetic scheme (arXiv:1901.00261).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this module.  The
product library (``paper_1901_00261_gb300``) never loads it and shares no code with it.

The arithmetic lives in ``gks_oracle.cpp`` (C++17, FP64, compiled without FMA
contraction so that x86 and Arm builds round identically).  This module compiles it on
first use and exposes thin ctypes wrappers.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gks_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgks_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, -O2, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            c_int, c_double, c_void = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            L.orc_set_threads.argtypes = [c_int]
            L.orc_get_threads.restype = c_int
            L.orc_linear_weights.argtypes = [c_int, dp]
            L.orc_linear_weights.restype = c_int
            L.orc_candidate.argtypes = [c_int, dp]
            L.orc_candidate.restype = c_int
            L.orc_smoothness.argtypes = [dp, c_int]
            L.orc_smoothness.restype = c_double
            L.orc_weno_left.argtypes = [c_int, dp, c_double, dp]
            L.orc_weno_left.restype = c_int
            L.orc_weno_right.argtypes = [c_int, dp, c_double, dp]
            L.orc_weno_right.restype = c_int
            L.orc_tangential_weights.argtypes = [dp, dp, dp]
            L.orc_maxwell_moments.argtypes = [c_int, c_double, c_double, c_double, c_double,
                                              dp, dp, dp, dp, dp]
            L.orc_moment_max.argtypes = [c_int]
            L.orc_moment_max.restype = c_int
            L.orc_solve_coef.argtypes = [c_int, c_double, c_double, c_double, c_double,
                                         c_double, dp, dp]
            L.orc_moment_lin.argtypes = [c_int, c_double, c_double, c_double, c_double,
                                         c_double, dp, c_int, c_int, c_int, dp]
            L.orc_time_integrals.argtypes = [c_double, c_double, dp, dp]
            L.orc_eigvecs.argtypes = [c_int, c_double, dp, dp]
            L.orc_point.argtypes = [c_int, c_double, c_double, c_double, c_int, c_int, c_int,
                                    dp, c_double, dp]
            L.orc_point.restype = c_int
            L.orc_create.argtypes = [c_int, c_int, c_double, c_double, c_double, c_int, c_int,
                                     c_int, c_int, c_double, c_double, c_double, c_double,
                                     c_double, c_int, c_int]
            L.orc_create.restype = c_void
            L.orc_destroy.argtypes = [c_void]
            L.orc_set_eq_mode.argtypes = [c_void, c_int]
            L.orc_set_char_mode.argtypes = [c_void, c_int]
            L.orc_set_tan_mode.argtypes = [c_void, c_int]
            L.orc_set_coef_mode.argtypes = [c_void, c_int]
            L.orc_set_coef_mode.restype = c_int
            L.orc_set_walls.argtypes = [c_void, dp, dp]
            L.orc_set_walls.restype = c_int
            L.orc_iso_ghost.argtypes = [c_void, c_int, c_int, c_int, dp, dp]
            L.orc_tan_weno.argtypes = [dp, c_int, c_int, c_double, dp]
            L.orc_tan_weno.restype = c_double
            L.orc_set_state.argtypes = [c_void, dp, dp, dp]
            L.orc_get_state.argtypes = [c_void, dp, dp, dp]
            L.orc_step.argtypes = [c_void, c_double]
            L.orc_step.restype = c_int
            L.orc_max_wavespeed.argtypes = [c_void]
            L.orc_max_wavespeed.restype = c_double
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def linear_weights(order: int) -> np.ndarray:
    """[3, 8]: interface value, d/ds and d2/ds2 weights of the compact linear reconstruction
    against (W_{i-1..i+2}, dx W'_{i-1..i+2}) (Sec. 3.1)."""
    out = np.zeros((3, 8))
    if lib().orc_linear_weights(order, _p(out)) != 0:
        raise ValueError("order must be 6 or 8")
    return out


def candidate(k: int):
    """Candidate polynomial k (0..6, 7 = the cubic w~1) of Sec. 3.3 as a [5, 8] matrix of
    coefficients of s^p (origin at the centre of cell i, unit cell) and its degree."""
    out = np.zeros((5, 8))
    deg = lib().orc_candidate(k, _p(out))
    return out, deg


def smoothness(c, deg: int) -> float:
    c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(-1)[:8])
    buf = np.zeros(8)
    buf[: c.size] = c
    return float(lib().orc_smoothness(_p(buf), int(deg)))


def weno_left(order: int, in8, eps: float = 1e-6):
    """Returns (value, d/ds, delta[7], beta[7]) of the WENO-Z left state (Sec. 3.3)."""
    x = np.ascontiguousarray(np.asarray(in8, dtype=np.float64))
    out = np.zeros(16)
    lib().orc_weno_left(order, _p(x), eps, _p(out))
    return out[0], out[1], out[2:9].copy(), out[9:16].copy()


def weno_right(order: int, in8, eps: float = 1e-6):
    x = np.ascontiguousarray(np.asarray(in8, dtype=np.float64))
    out = np.zeros(2)
    lib().orc_weno_right(order, _p(x), eps, _p(out))
    return out[0], out[1]


def tan_weno(q5, g: int, der: int = 0, eps: float = 1e-6):
    """Tangential WENO-Z (reading R9's variant) of 5 segment averages at Gauss point g:
    (value or d/ds at s_g, the rule's 3 linear weights)."""
    q = np.ascontiguousarray(np.asarray(q5, dtype=np.float64))
    d = np.zeros(3)
    v = lib().orc_tan_weno(_p(q), int(g), int(der), float(eps), _p(d))
    return v, d


def tangential_weights():
    """([3 gauss][3 derivs][5], gauss nodes, gauss weights) of the tangential quartic."""
    w = np.zeros((3, 3, 5))
    gs = np.zeros(3)
    gw = np.zeros(3)
    lib().orc_tangential_weights(_p(w), _p(gs), _p(gw))
    return w, gs, gw


def maxwell_moments(dim: int, K: float, U: float, V: float, lam: float):
    L = lib()
    nu, nv, nk = L.orc_moment_max(0) + 1, L.orc_moment_max(1) + 1, L.orc_moment_max(2) + 1
    mu, mup, mun = np.zeros(nu), np.zeros(nu), np.zeros(nu)
    mv, mx = np.zeros(nv), np.zeros(nk)
    L.orc_maxwell_moments(dim, K, U, V, lam, _p(mu), _p(mup), _p(mun), _p(mv), _p(mx))
    return dict(mu=mu, mup=mup, mun=mun, mv=mv, mx=mx)


def solve_coef(dim: int, K: float, rho: float, U: float, V: float, lam: float, b) -> np.ndarray:
    bb = np.ascontiguousarray(np.asarray(b, dtype=np.float64))
    a = np.zeros(dim + 2)
    lib().orc_solve_coef(dim, K, rho, U, V, lam, _p(bb), _p(a))
    return a


def moment_lin(dim, K, rho, U, V, lam, c, a=0, b=0, space=0) -> np.ndarray:
    cc = np.ascontiguousarray(np.asarray(c, dtype=np.float64))
    out = np.zeros(dim + 2)
    lib().orc_moment_lin(dim, K, rho, U, V, lam, _p(cc), a, b, space, _p(out))
    return out


def time_integrals(d: float, tau: float):
    e0 = ctypes.c_double()
    e1 = ctypes.c_double()
    lib().orc_time_integrals(d, tau, ctypes.byref(e0), ctypes.byref(e1))
    return e0.value, e1.value


def eigvecs(dim: int, gamma: float, W) -> np.ndarray:
    w = np.ascontiguousarray(np.asarray(W, dtype=np.float64))
    R = np.zeros((dim + 2, dim + 2))
    lib().orc_eigvecs(dim, gamma, _p(w), _p(R))
    return R


POINT_FIELDS = ("W0", "W0x", "W0y", "W0xx", "W0xy", "W0yy", "Wl", "Wlx", "Wly", "Wr", "Wrx", "Wry")


def point(dim: int, gamma: float, mu: float, Pr: float, fields: dict, dt: float,
          tau_mode: int = 0, flux_mode: int = 0, coef_mode: int = 0) -> dict:
    # (the equilibrium value is always the collision of Wl and Wr here; pass Wl = Wr = W0
    # for the linear scheme)
    """Gas-kinetic evaluation at one interface point (Eq. 3rd-simplify-flux)."""
    pin = np.zeros((12, 4))
    for i, name in enumerate(POINT_FIELDS):
        if name in fields:
            v = np.asarray(fields[name], dtype=np.float64)
            pin[i, : v.size] = v
    out = np.zeros((5, 4))
    rc = lib().orc_point(dim, gamma, mu, Pr, tau_mode, flux_mode, coef_mode, _p(pin), dt, _p(out))
    if rc != 0:
        raise ValueError("non-physical state")
    n = dim + 2
    return dict(F=out[0, :n].copy(), Ft=out[1, :n].copy(), W0=out[2, :n].copy(),
                Wt=out[3, :n].copy(), Wtt=out[4, :n].copy())


class Solver:
    """The whole two-stage scheme on a 1D (ny == 1) or 2D grid.

    State arrays are C-contiguous [nvar][ny][nx] FP64: conservative cell averages W and
    cell-averaged gradients Wx (and Wy in 2D)."""

    def __init__(self, nx: int, ny: int, gamma: float = 1.4, mu: float = 0.0, Pr: float = 1.0,
                 order: int = 6, recon: int = 0, bc_x: int = 0, bc_y: int = 0,
                 x0: float = 0.0, x1: float = 1.0, y0: float = 0.0, y1: float = 1.0,
                 weno_eps: float = 1e-6, tau_mode: int = 0, flux_mode: int = 0,
                 eq_mode: int = 1, char_mode: int = 0, tan_mode: int = 0,
                 wall_T=(1.0, 1.0, 1.0, 1.0), wall_u=(0.0, 0.0, 0.0, 0.0), coef_mode: int = 0):
        self.nx, self.ny = nx, ny
        self.dim = 2 if ny > 1 else 1
        self.nv = self.dim + 2
        self._h = lib().orc_create(nx, ny, gamma, mu, Pr, order, recon, bc_x, bc_y,
                                   x0, x1, y0, y1, weno_eps, tau_mode, flux_mode)
        if not self._h:
            raise ValueError("invalid oracle parameters")
        lib().orc_set_eq_mode(self._h, int(eq_mode))
        lib().orc_set_char_mode(self._h, int(char_mode))
        lib().orc_set_tan_mode(self._h, int(tan_mode))
        if lib().orc_set_coef_mode(self._h, int(coef_mode)) != 0:
            lib().orc_destroy(self._h)
            self._h = None
            raise ValueError("coef_mode must be 0 or 1; 1 needs mu = 0 and tau_mode 0")
        wt = np.ascontiguousarray(wall_T, dtype=np.float64)
        wu = np.ascontiguousarray(wall_u, dtype=np.float64)
        if lib().orc_set_walls(self._h, _p(wt), _p(wu)) != 0:
            lib().orc_destroy(self._h)
            self._h = None
            raise ValueError("a moving isothermal wall meets a reflecting wall")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    @property
    def shape(self):
        return (self.nv, self.ny, self.nx)

    def set_state(self, W, Wx, Wy=None):
        W = np.ascontiguousarray(W, dtype=np.float64).reshape(self.shape)
        Wx = np.ascontiguousarray(Wx, dtype=np.float64).reshape(self.shape)
        if self.dim == 2:
            Wy = np.ascontiguousarray(Wy, dtype=np.float64).reshape(self.shape)
            lib().orc_set_state(self._h, _p(W), _p(Wx), _p(Wy))
        else:
            lib().orc_set_state(self._h, _p(W), _p(Wx), None)

    def get_state(self):
        W = np.zeros(self.shape)
        Wx = np.zeros(self.shape)
        if self.dim == 2:
            Wy = np.zeros(self.shape)
            lib().orc_get_state(self._h, _p(W), _p(Wx), _p(Wy))
            return W, Wx, Wy
        lib().orc_get_state(self._h, _p(W), _p(Wx), None)
        return W, Wx, None

    def step(self, dt: float) -> None:
        rc = lib().orc_step(self._h, float(dt))
        if rc != 0:
            raise RuntimeError(f"oracle step failed ({rc})")

    def max_wavespeed(self) -> float:
        return float(lib().orc_max_wavespeed(self._h))

    def iso_ghost(self, axis: int, side: int, normal: bool, w, d):
        """Ghost of an isothermal wall (bc 3) for the mirror cell's conservative values w and
        their derivatives d along the stencil (across the wall when normal).  axis 1 = x,
        2 = y; side 0 = the low wall, 1 = the high one.  Returns (w_ghost, d_ghost)."""
        w = np.array(w, dtype=np.float64)
        d = np.array(d, dtype=np.float64)
        if lib().orc_iso_ghost(self._h, int(axis), int(side), int(bool(normal)), _p(w), _p(d)) != 0:
            raise ValueError("bad wall")
        return w, d
