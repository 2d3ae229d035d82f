"""Seeded synthetic inputs: initial cell averages and cell-averaged gradients.

This module holds none of the scheme's arithmetic.  It turns point-wise initial
conditions into the state the scheme evolves -- conservative cell averages W and
cell-averaged gradients W_x (W_y) -- and evaluates exact solutions for error norms.
Both the GPU library's tests/benchmark and the CPU oracle's tests take their inputs
from here.

Layout of every state array: C-contiguous float64 ``[nvar][ny][nx]`` with
nvar = 3 (1D: rho, rho U, rho E) or 4 (2D: rho, rho U, rho V, rho E).

Cell averages use Gauss-Legendre quadrature (exact antiderivatives where the profile
has one).  The averaged gradient of a cell is the difference of the face (line)
averages of W divided by the cell size (Gauss formula); a discontinuity lying exactly
on a face is excluded by taking the one-sided value from inside the cell.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAUSS6_X, GAUSS6_W = np.polynomial.legendre.leggauss(6)
GAUSS10_X, GAUSS10_W = np.polynomial.legendre.leggauss(10)


# ---------------------------------------------------------------------------
# Counter-based random numbers: splitmix64 (G. Steele, D. Lea, C. Flood,
# "Fast splittable pseudorandom number generators", OOPSLA 2014).
# ---------------------------------------------------------------------------
_M64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    z = (x + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def uniform01(seed: int, counter: int) -> float:
    """U[0,1) from the 53 top bits of splitmix64(seed * 2^32 + counter)."""
    return (splitmix64(((seed & 0xFFFFFFFF) << 32) + counter) >> 11) * (1.0 / (1 << 53))


def uniform01_array(seed: int, n: int) -> np.ndarray:
    """Vectorised splitmix64 stream: element k = uniform01(seed, k)."""
    with np.errstate(over="ignore"):
        x = (np.uint64((seed & 0xFFFFFFFF) << 32) + np.arange(n, dtype=np.uint64))
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


# ---------------------------------------------------------------------------
# Primitive <-> conservative
# ---------------------------------------------------------------------------
def conservative_1d(rho, u, p, gamma):
    return np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])


def conservative_2d(rho, u, v, p, gamma):
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


@dataclass
class State:
    """Initial state of one problem plus everything needed to run it."""
    W: np.ndarray
    Wx: np.ndarray
    Wy: np.ndarray | None
    nx: int
    ny: int
    gamma: float
    x0: float
    x1: float
    y0: float = 0.0
    y1: float = 1.0
    bc_x: int = 0          # 0 periodic, 1 transmissive, 2 reflecting wall, 3 isothermal wall
    bc_y: int = 0
    mu: float = 0.0
    Pr: float = 1.0
    order: int = 6
    recon: int = 0         # 0 linear, 1 WENO-Z
    t_end: float = 0.0
    name: str = ""
    meta: dict = field(default_factory=dict)
    # isothermal no-slip walls (bc 3): temperature p/rho and tangential velocity of the walls
    # at x0, x1, y0, y1
    wall_T: tuple = (1.0, 1.0, 1.0, 1.0)
    wall_u: tuple = (0.0, 0.0, 0.0, 0.0)

    @property
    def dx(self):
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self):
        return (self.y1 - self.y0) / self.ny


# ---------------------------------------------------------------------------
# 1D profiles given piecewise: list of (x_left, x_right, f) with f(x) -> (rho, u, p)
# ---------------------------------------------------------------------------
def _piece_at(pieces, x, inside_of):
    """Piece containing x, choosing the one on the side of the cell centre inside_of
    when x is a breakpoint."""
    for a, b, f in pieces:
        if a <= x <= b:
            if x == a and inside_of < a:
                continue
            if x == b and inside_of > b:
                continue
            return f
    raise ValueError(f"x={x} outside profile")


def cell_state_1d(pieces, N, x0, x1, gamma):
    """Exact-to-quadrature cell averages and averaged slopes of conservative variables."""
    dx = (x1 - x0) / N
    W = np.zeros((3, 1, N))
    Wx = np.zeros((3, 1, N))
    breaks = sorted({a for a, _, _ in pieces} | {b for _, b, _ in pieces})
    for i in range(N):
        a, b = x0 + i * dx, x0 + (i + 1) * dx
        pts = [a] + [q for q in breaks if a < q < b] + [b]
        acc = np.zeros(3)
        for lo, hi in zip(pts[:-1], pts[1:]):
            mid = 0.5 * (lo + hi)
            f = _piece_at(pieces, mid, mid)
            xs = mid + 0.5 * (hi - lo) * GAUSS10_X
            rho, u, p = f(xs)
            acc += conservative_1d(rho, u, p, gamma) @ GAUSS10_W * 0.5 * (hi - lo)
        W[:, 0, i] = acc / dx
        c = 0.5 * (a + b)
        fr = _piece_at(pieces, b, c)
        fl = _piece_at(pieces, a, c)
        wr = conservative_1d(*[np.asarray(q, dtype=float) for q in fr(np.array([b]))], gamma)[:, 0]
        wl = conservative_1d(*[np.asarray(q, dtype=float) for q in fl(np.array([a]))], gamma)[:, 0]
        Wx[:, 0, i] = (wr - wl) / dx
    return W, Wx


def density_wave_1d(N: int, t: float = 0.0, gamma: float = 1.4, order: int = 6, recon: int = 0,
                    x0: float = 0.0, x1: float = 2.0) -> State:
    """rho = 1 + 0.2 sin(pi (x - t)), U = 1, p = 1 on periodic [0, 2] (Sec. 4.1).
    Exact averages from the antiderivative."""
    dx = (x1 - x0) / N
    xl = x0 + dx * np.arange(N)
    xr = xl + dx
    # average of sin(pi (x - t)) over the cell
    avg_sin = (np.cos(np.pi * (xl - t)) - np.cos(np.pi * (xr - t))) / (np.pi * dx)
    rho_avg = 1.0 + 0.2 * avg_sin
    W = np.zeros((3, 1, N))
    W[0, 0] = rho_avg
    W[1, 0] = rho_avg                      # U = 1
    W[2, 0] = 1.0 / (gamma - 1.0) + 0.5 * rho_avg
    rho_r = 1.0 + 0.2 * np.sin(np.pi * (xr - t))
    rho_l = 1.0 + 0.2 * np.sin(np.pi * (xl - t))
    drho = (rho_r - rho_l) / dx
    Wx = np.zeros((3, 1, N))
    Wx[0, 0] = drho
    Wx[1, 0] = drho
    Wx[2, 0] = 0.5 * drho
    return State(W, Wx, None, N, 1, gamma, x0, x1, bc_x=0, order=order, recon=recon,
                 t_end=2.0, name="density_wave_1d")


def density_wave_exact_rho(N: int, t: float, x0: float = 0.0, x1: float = 2.0) -> np.ndarray:
    dx = (x1 - x0) / N
    xl = x0 + dx * np.arange(N)
    xr = xl + dx
    return 1.0 + 0.2 * (np.cos(np.pi * (xl - t)) - np.cos(np.pi * (xr - t))) / (np.pi * dx)


def riemann_1d(N: int, left, right, x0: float, x1: float, xjump: float, gamma: float = 1.4,
               order: int = 8, recon: int = 1, t_end: float = 0.2, name: str = "riemann") -> State:
    """Piecewise-constant Riemann data (rho, u, p) | (rho, u, p), transmissive ends."""
    def const(s):
        return lambda x: tuple(np.full_like(np.asarray(x, dtype=float), q) for q in s)
    pieces = [(x0, xjump, const(left)), (xjump, x1, const(right))]
    W, Wx = cell_state_1d(pieces, N, x0, x1, gamma)
    return State(W, Wx, None, N, 1, gamma, x0, x1, bc_x=1, order=order, recon=recon,
                 t_end=t_end, name=name, meta=dict(left=tuple(left), right=tuple(right), xjump=xjump))


def sod_1d(N: int = 1000, gamma: float = 1.4, order: int = 8, recon: int = 1) -> State:
    """Sod tube (1, 0, 1) | (0.125, 0, 0.1) on [0, 1], jump at 0.5, t = 0.2."""
    return riemann_1d(N, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.0, 1.0, 0.5, gamma, order, recon,
                      0.2, "sod_1d")


def shu_osher_1d(N: int = 400, gamma: float = 1.4, order: int = 8, recon: int = 1) -> State:
    """Shock / density-wave interaction on [-5, 5]: (3.857143, 2.629369, 10.33333) for
    x < -4, else (1 + 0.2 sin 5x, 0, 1); transmissive ends; t = 1.8."""
    x0, x1 = -5.0, 5.0

    def left(x):
        x = np.asarray(x, dtype=float)
        return np.full_like(x, 3.857143), np.full_like(x, 2.629369), np.full_like(x, 10.33333)

    def right(x):
        x = np.asarray(x, dtype=float)
        return 1.0 + 0.2 * np.sin(5.0 * x), np.zeros_like(x), np.ones_like(x)

    W, Wx = cell_state_1d([(x0, -4.0, left), (-4.0, x1, right)], N, x0, x1, gamma)
    return State(W, Wx, None, N, 1, gamma, x0, x1, bc_x=1, order=order, recon=recon,
                 t_end=1.8, name="shu_osher_1d")


def acoustic_1d(N: int = 40, gamma: float = 1.4, order: int = 8, recon: int = 0) -> State:
    """Small-amplitude acoustic wave of Sec. 4.3 on periodic [0, 1/3]."""
    eps, om, rinf, pinf = 1e-5, 6.0 * math.pi, 1.1771, 101325.0
    ainf = math.sqrt(gamma * pinf / rinf)

    def prof(x):
        x = np.asarray(x, dtype=float)
        rho = rinf + eps * rinf * np.cos(2 * om * x)
        u = eps * ainf * np.cos(om * x)
        p = pinf * (rho / rinf) ** gamma
        return rho, u, p

    W, Wx = cell_state_1d([(0.0, 1.0 / 3.0, prof)], N, 0.0, 1.0 / 3.0, gamma)
    return State(W, Wx, None, N, 1, gamma, 0.0, 1.0 / 3.0, bc_x=0, order=order, recon=recon,
                 t_end=0.01, name="acoustic_1d")


def wall_impact_1d(N: int, u0: float = 0.5, rho: float = 1.0, p: float = 1.0,
                   gamma: float = 1.4, order: int = 8, recon: int = 1) -> State:
    """Uniform flow (rho, u0, p) in a tube [0, 1] closed by reflecting walls at both ends.
    Until the waves from the two walls meet, the solution near x = 1 is the Riemann problem
    of (rho, u0, p) against its mirror image (rho, -u0, p) (two shocks; the wall keeps the
    middle state at rest), and near x = 0 the one of (rho, -u0, p) against (rho, u0, p)
    (two rarefactions).  t_end = 0.2 keeps the two wave systems apart for u0 <= 1."""
    W, Wx = cell_state_1d([(0.0, 1.0, lambda x: (np.full_like(x, rho), np.full_like(x, u0),
                                                  np.full_like(x, p)))], N, 0.0, 1.0, gamma)
    return State(W, Wx, None, N, 1, gamma, 0.0, 1.0, bc_x=2, order=order, recon=recon,
                 t_end=0.2, name="wall_impact_1d", meta=dict(state=(rho, u0, p)))


# ---------------------------------------------------------------------------
# 2D
# ---------------------------------------------------------------------------
def _cell_state_2d(point_fn, nx, ny, x0, x1, y0, y1, gamma, rows=None):
    """Cell averages (6x6 Gauss) and averaged gradients (6-point Gauss on faces) of a smooth
    point function point_fn(x, y) -> conservative [4, ...]."""
    dx, dy = (x1 - x0) / nx, (y1 - y0) / ny
    xc = x0 + dx * (np.arange(nx) + 0.5)
    yc = y0 + dy * (np.arange(ny) + 0.5)
    W = np.zeros((4, ny, nx))
    Wx = np.zeros((4, ny, nx))
    Wy = np.zeros((4, ny, nx))
    gx = 0.5 * GAUSS6_X
    gw = 0.5 * GAUSS6_W
    for a in range(6):
        ys = yc + gx[a] * dy
        Y = ys[:, None]
        # face line averages in y at x faces, and the cell average
        Wx += gw[a] * (point_fn(xc[None, :] + 0.5 * dx, Y) - point_fn(xc[None, :] - 0.5 * dx, Y)) / dx
        for b in range(6):
            xs = xc + gx[b] * dx
            W += gw[a] * gw[b] * point_fn(xs[None, :], Y)
    for b in range(6):
        xs = xc + gx[b] * dx
        X = xs[None, :]
        Wy += gw[b] * (point_fn(X, yc[:, None] + 0.5 * dy) - point_fn(X, yc[:, None] - 0.5 * dy)) / dy
    return W, Wx, Wy


def vortex_point(x, y, t=0.0, gamma=1.4, beta=5.0, L=10.0, xc=5.0, yc=5.0):
    """Isentropic vortex of strength beta on the background (1, 1, 1, 1), centre
    translated by (t, t), nearest periodic image on [0, L]^2."""
    xb = np.mod(x - xc - t + 0.5 * L, L) - 0.5 * L
    yb = np.mod(y - yc - t + 0.5 * L, L) - 0.5 * L
    r2 = xb * xb + yb * yb
    e = np.exp(0.5 * (1.0 - r2))
    u = 1.0 - beta / (2 * math.pi) * e * yb
    v = 1.0 + beta / (2 * math.pi) * e * xb
    T = 1.0 - (gamma - 1.0) * beta * beta * e * e / (8.0 * gamma * math.pi ** 2)
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho * T
    return conservative_2d(rho, u, v, p, gamma)


def isentropic_vortex_2d(n: int, t: float = 0.0, gamma: float = 1.4, order: int = 8,
                         recon: int = 0, ny: int | None = None) -> State:
    ny = n if ny is None else ny
    W, Wx, Wy = _cell_state_2d(lambda x, y: vortex_point(x, y, t, gamma), n, ny, 0.0, 10.0,
                               0.0, 10.0 * ny / n, gamma)
    return State(W, Wx, Wy, n, ny, gamma, 0.0, 10.0, 0.0, 10.0 * ny / n, 0, 0, order=order,
                 recon=recon, t_end=10.0, name="isentropic_vortex_2d")


def box_pulse_point(x, y, gamma=1.4):
    """Smooth pressure and density pulse off the centre of [0, 1]^2 with a swirl and a
    uniform drift, so that every wall sees a normal and a tangential velocity."""
    r2 = (x - 0.35) ** 2 + (y - 0.6) ** 2
    g = np.exp(-r2 / 0.02)
    rho = 1.0 + 0.3 * g
    p = 1.0 + 0.5 * g
    u = 0.2 - 2.0 * (y - 0.6) * g
    v = -0.1 + 2.0 * (x - 0.35) * g
    return conservative_2d(rho, u, v, p, gamma)


def box_pulse_2d(n: int, ny: int | None = None, gamma: float = 1.4, mu: float = 0.0,
                 Pr: float = 1.0, order: int = 8, recon: int = 0, bc_x: int = 2,
                 bc_y: int = 2) -> State:
    """box_pulse_point on [0, 1] x [0, ny/n] (reflecting walls by default)."""
    ny = n if ny is None else ny
    W, Wx, Wy = _cell_state_2d(lambda x, y: box_pulse_point(x, y, gamma), n, ny, 0.0, 1.0,
                               0.0, ny / n, gamma)
    return State(W, Wx, Wy, n, ny, gamma, 0.0, 1.0, 0.0, ny / n, bc_x, bc_y, mu=mu, Pr=Pr,
                 order=order, recon=recon, t_end=0.5, name="box_pulse_2d")


def shear_wave_2d(nx: int, ny: int, U0: float = 0.01, mu: float = 0.01, Pr: float = 0.72,
                  gamma: float = 1.4, order: int = 8, recon: int = 0) -> State:
    """Transverse viscous shear wave on periodic [0, nx/ny] x [0, 1]: rho = 1, p = 1/gamma,
    u = U0 sin(2 pi y), v = 0.  Linearised Navier-Stokes: u decays as exp(-mu/rho (2 pi)^2 t)
    with the pressure uniform (viscous heating enters at order U0^2)."""
    k = 2.0 * math.pi

    def pt(x, y):
        u = U0 * np.sin(k * y) + 0.0 * x
        one = np.ones_like(u)
        return conservative_2d(one, u, 0.0 * u, one / gamma, gamma)
    W, Wx, Wy = _cell_state_2d(pt, nx, ny, 0.0, nx / ny, 0.0, 1.0, gamma)
    return State(W, Wx, Wy, nx, ny, gamma, 0.0, nx / ny, 0.0, 1.0, 0, 0, mu=mu, Pr=Pr,
                 order=order, recon=recon, t_end=0.5, name="shear_wave_2d",
                 meta=dict(U0=U0, k=k))


def entropy_wave_2d(nx: int, ny: int, delta: float = 0.01, mu: float = 0.01, Pr: float = 0.72,
                    gamma: float = 1.4, order: int = 8, recon: int = 0) -> State:
    """Static entropy (temperature) wave on periodic [0, nx/ny] x [0, 1]: rho = 1 +
    delta sin(2 pi y), p = 1/gamma, u = v = 0.  Linearised Navier-Stokes: the entropy
    perturbation p'/p - gamma rho'/rho decays by heat conduction as exp(-chi (2 pi)^2 t),
    chi = kappa / (rho c_p) = mu / (rho Pr), up to corrections of second order in chi."""
    k = 2.0 * math.pi

    def pt(x, y):
        rho = 1.0 + delta * np.sin(k * y) + 0.0 * x
        zero = 0.0 * rho
        return conservative_2d(rho, zero, zero, np.full_like(rho, 1.0 / gamma), gamma)
    W, Wx, Wy = _cell_state_2d(pt, nx, ny, 0.0, nx / ny, 0.0, 1.0, gamma)
    return State(W, Wx, Wy, nx, ny, gamma, 0.0, nx / ny, 0.0, 1.0, 0, 0, mu=mu, Pr=Pr,
                 order=order, recon=recon, t_end=0.5, name="entropy_wave_2d", meta=dict(k=k))


def entropy_wave_amplitude(st, W) -> float:
    """Amplitude of the sin(2 pi y) mode of the entropy perturbation p'/p0 - gamma rho'/rho0
    of the cell averages W (rho0 = 1, p0 = 1/gamma), projected as in shear_wave_amplitude."""
    g = st.gamma
    rho = W[0]
    u, v = W[1] / rho, W[2] / rho
    p = (g - 1.0) * (W[3] - 0.5 * rho * (u * u + v * v))
    s_prime = (p - 1.0 / g) * g - g * (rho - 1.0)
    k, h = st.meta["k"], (st.y1 - st.y0) / st.ny
    yc = st.y0 + h * (np.arange(st.ny) + 0.5)
    s = (np.cos(k * (yc - h / 2)) - np.cos(k * (yc + h / 2))) / (k * h)
    return float((s_prime.mean(axis=1) * s).sum() / (s * s).sum())


def shear_wave_amplitude(st, W) -> float:
    """Amplitude of the sin(2 pi y) mode of the x-momentum cell averages W[1] (projection on
    the cell averages of sin(2 pi y))."""
    k, h = st.meta["k"], (st.y1 - st.y0) / st.ny
    yc = st.y0 + h * (np.arange(st.ny) + 0.5)
    s = (np.cos(k * (yc - h / 2)) - np.cos(k * (yc + h / 2))) / (k * h)
    return float((W[1].mean(axis=1) * s).sum() / (s * s).sum())


def vortex_exact_avg(n: int, t: float, gamma: float = 1.4, ny: int | None = None) -> np.ndarray:
    ny = n if ny is None else ny
    W, _, _ = _cell_state_2d(lambda x, y: vortex_point(x, y, t, gamma), n, ny, 0.0, 10.0,
                             0.0, 10.0 * ny / n, gamma)
    return W


def shear_layer_2d(n: int, seed: int = 0, gamma: float = 1.4, mu: float = 1e-4, Pr: float = 0.72,
                   order: int = 8, recon: int = 1, noise: float = 1e-3) -> State:
    """Double shear layer on periodic [0,1]^2: rho = 1, p = 1/gamma, u = 0.5 tanh((y-0.25)/0.01)
    for y <= 0.5 else -0.5 tanh((y-0.75)/0.01), v = 0.01 sin(4 pi x) + noise * U(-1,1) per cell
    (splitmix64 stream, cell-constant)."""
    nx = ny = n
    dx = dy = 1.0 / n
    nz = noise * (2.0 * uniform01_array(seed, nx * ny).reshape(ny, nx) - 1.0)
    xc = dx * (np.arange(nx) + 0.5)
    yc = dy * (np.arange(ny) + 0.5)
    J, I = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")

    def pfn_cell(xoff, yoff):
        x = xc[None, :] + xoff * dx
        y = yc[:, None] + yoff * dy
        yy = np.broadcast_to(y, (ny, nx))
        xx = np.broadcast_to(x, (ny, nx))
        # piece chosen by the cell centre so that the (smooth) tanh profile is per-cell
        lower = (yc[:, None] <= 0.5)
        u = np.where(lower, 0.5 * np.tanh((yy - 0.25) / 0.01), -0.5 * np.tanh((yy - 0.75) / 0.01))
        v = 0.01 * np.sin(4.0 * math.pi * xx) + nz
        rho = np.ones_like(u)
        p = np.full_like(u, 1.0 / gamma)
        return conservative_2d(rho, u, v, p, gamma)

    gx = 0.5 * GAUSS6_X
    gw = 0.5 * GAUSS6_W
    W = np.zeros((4, ny, nx))
    Wx = np.zeros((4, ny, nx))
    Wy = np.zeros((4, ny, nx))
    for a in range(6):
        Wx += gw[a] * (pfn_cell(0.5, gx[a]) - pfn_cell(-0.5, gx[a])) / dx
        Wy += gw[a] * (pfn_cell(gx[a], 0.5) - pfn_cell(gx[a], -0.5)) / dy
        for b in range(6):
            W += gw[a] * gw[b] * pfn_cell(gx[b], gx[a])
    del J, I
    return State(W, Wx, Wy, nx, ny, gamma, 0.0, 1.0, 0.0, 1.0, 0, 0, mu=mu, Pr=Pr, order=order,
                 recon=recon, t_end=1.0, name="shear_layer_2d")


# ---------------------------------------------------------------------------
# Flows between isothermal no-slip walls
# ---------------------------------------------------------------------------
def couette_profile(y, U, T0, Pr, gamma):
    """Plane Couette flow between walls at y = 0 (at rest) and y = 1 (moving at U), both at
    temperature T0 = p/rho, with constant viscosity and Prandtl number: u = U y, uniform p,
    and the viscous heating k T'' + mu u'^2 = 0 with k = mu c_p / Pr, c_p = gamma/(gamma - 1)
    (gas constant 1), i.e. T = T0 + Pr U^2 / (2 c_p) y (1 - y).  Returns (u, T)."""
    cp = gamma / (gamma - 1.0)
    return U * y, T0 + Pr * U * U / (2.0 * cp) * y * (1.0 - y)


def couette_2d(ny: int, nx: int = 5, U: float = 0.2, mu: float = 0.02, Pr: float = 0.72,
               gamma: float = 1.4, order: int = 8, recon: int = 0, walls: str = "y") -> State:
    """Steady plane Couette flow (couette_profile, p = 1/gamma, T0 = 1/gamma) as the initial
    state.  walls "y": periodic in x on [0, nx/ny], isothermal walls at y = 0, 1, the upper
    one moving at U along x.  walls "x": the same flow turned by a quarter: walls at x = 0, 1,
    the one at x = 1 moving at U along y, periodic in y on [0, nx/ny] (nx, ny swap roles)."""
    T0 = 1.0 / gamma

    def pt(s):
        u, T = couette_profile(s, U, T0, Pr, gamma)
        return u, T

    if walls == "y":
        def pfn(x, y):
            u, T = pt(y)
            p = np.full(np.broadcast(x, y).shape, 1.0 / gamma)
            return conservative_2d(p / T + 0 * x, u + 0 * x, 0.0 * (x + y), p, gamma)
        W, Wx, Wy = _cell_state_2d(pfn, nx, ny, 0.0, nx / ny, 0.0, 1.0, gamma)
        return State(W, Wx, Wy, nx, ny, gamma, 0.0, nx / ny, 0.0, 1.0, 0, 3, mu=mu, Pr=Pr,
                     order=order, recon=recon, t_end=5.0, name="couette_2d",
                     meta=dict(U=U, T0=T0), wall_T=(T0,) * 4, wall_u=(0.0, 0.0, 0.0, U))

    def pfn(x, y):
        v, T = pt(x)
        p = np.full(np.broadcast(x, y).shape, 1.0 / gamma)
        return conservative_2d(p / T + 0 * y, 0.0 * (x + y), v + 0 * y, p, gamma)
    W, Wx, Wy = _cell_state_2d(pfn, ny, nx, 0.0, 1.0, 0.0, nx / ny, gamma)
    return State(W, Wx, Wy, ny, nx, gamma, 0.0, 1.0, 0.0, nx / ny, 3, 0, mu=mu, Pr=Pr,
                 order=order, recon=recon, t_end=5.0, name="couette_2d_x",
                 meta=dict(U=U, T0=T0), wall_T=(T0,) * 4, wall_u=(0.0, U, 0.0, 0.0))


def heat_conduction_1d(N: int, TL: float = 0.6, TR: float = 0.8, mu: float = 0.02,
                       Pr: float = 0.72, gamma: float = 1.4, order: int = 8,
                       recon: int = 0) -> State:
    """Gas at rest between isothermal walls at x = 0 (temperature TL = p/rho) and x = 1 (TR),
    in its steady state with constant conductivity: T linear, p = 1/gamma, rho = p/T."""
    p = 1.0 / gamma

    def f(x):
        T = TL + (TR - TL) * x
        return p / T, 0.0 * x, np.full_like(x, p)
    W, Wx = cell_state_1d([(0.0, 1.0, f)], N, 0.0, 1.0, gamma)
    return State(W, Wx, None, N, 1, gamma, 0.0, 1.0, bc_x=3, mu=mu, Pr=Pr, order=order,
                 recon=recon, t_end=5.0, name="heat_conduction_1d", meta=dict(TL=TL, TR=TR),
                 wall_T=(TL, TR, 1.0, 1.0))


def lid_cavity_2d(n: int, U: float = 0.15, Re: float = 1000.0, gamma: float = 1.4,
                  Pr: float = 0.72, order: int = 8, recon: int = 1) -> State:
    """Lid-driven cavity on [0,1]^2 (Sec. 5): gas at rest, rho = 1, p = 1/gamma (T = p/rho on
    every wall), isothermal no-slip walls on all four sides, the upper one moving at U along
    x; mu = rho U L / Re."""
    T0 = 1.0 / gamma

    def pfn(x, y):
        one = np.ones(np.broadcast(x, y).shape)
        return conservative_2d(one, 0.0 * one, 0.0 * one, one / gamma, gamma)
    W, Wx, Wy = _cell_state_2d(pfn, n, n, 0.0, 1.0, 0.0, 1.0, gamma)
    return State(W, Wx, Wy, n, n, gamma, 0.0, 1.0, 0.0, 1.0, 3, 3, mu=U / Re, Pr=Pr,
                 order=order, recon=recon, t_end=1.0, name="lid_cavity_2d",
                 meta=dict(U=U, Re=Re), wall_T=(T0,) * 4, wall_u=(0.0, 0.0, 0.0, U))


# ---------------------------------------------------------------------------
# Batched mixed workload: 1D Riemann problems and 2D vortices of uneven sizes.
# ---------------------------------------------------------------------------
@dataclass
class ProblemSpec:
    kind: str          # "riemann_1d" or "vortex_2d"
    n: int
    order: int
    left: tuple = ()
    right: tuple = ()


def batch_specs(count: int = 512, seed: int = 0, n1_range=(100, 20000), n2_range=(64, 1024)):
    """Problem s: even -> 1D Riemann, N log-uniform in n1_range, (rho, p) ~ U(0.1, 2) and
    u ~ U(-1, 1) per side; odd -> 2D vortex, side log-uniform in n2_range; order 6 or 8 from
    bit 1 of s."""
    specs = []
    for s in range(count):
        base = seed * 1_000_003 + s * 16
        r = [uniform01(base, k) for k in range(8)]
        order = 8 if (s >> 1) & 1 else 6
        if s % 2 == 0:
            lo, hi = n1_range
            n = int(round(math.exp(math.log(lo) + r[0] * (math.log(hi) - math.log(lo)))))
            left = (0.1 + 1.9 * r[1], -1.0 + 2.0 * r[2], 0.1 + 1.9 * r[3])
            right = (0.1 + 1.9 * r[4], -1.0 + 2.0 * r[5], 0.1 + 1.9 * r[6])
            specs.append(ProblemSpec("riemann_1d", n, order, left, right))
        else:
            lo, hi = n2_range
            n = int(round(math.exp(math.log(lo) + r[0] * (math.log(hi) - math.log(lo)))))
            specs.append(ProblemSpec("vortex_2d", n, order))
    return specs


def build_problem(spec: ProblemSpec) -> State:
    if spec.kind == "riemann_1d":
        return riemann_1d(spec.n, spec.left, spec.right, 0.0, 1.0, 0.5, 1.4, spec.order, 1, 0.1,
                          "riemann_1d")
    return isentropic_vortex_2d(spec.n, 0.0, 1.4, spec.order, 0)
