"""Pins of the oracle's isothermal no-slip walls (bc 3, reading R25: a ghost cell carries the
primitive state of the mirror cell inside with the same pressure, the velocity reflected
through the wall's (normal component negated, tangential u_t -> 2 u_w - u_t) and the
temperature p/rho reflected through the wall's, T -> 2 T_w - T).

1. The ghost's derivatives are those of the ghost field: finite differences of the mapped
   point field, across and along each of the four walls, against the oracle's derivative
   rule (a wrong sign on any variable's derivative fails).
2. Plane Couette flow (closed form: u linear, parabolic viscous-heating temperature, uniform
   pressure) stays on its exact profile within second-order errors, which fall by ~4 when
   the grid is refined twice; a dropped wall velocity or temperature, or a wrong-signed
   ghost slope, leaves an O(1) error.
3. Steady heat conduction between walls at two temperatures (1D): T linear.
4. The Couette flow turned by a quarter (walls normal to x) is, cell for cell, the turned
   result of the walls normal to y.
5. The lid-driven cavity with its lid reversed is the mirror image (x -> 1 - x, u -> -u) of
   the original, which ties the four walls and corners to one another.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1901_00261_gb300 import inputs


def _solver(st, **kw):
    O = oracle.Solver(st.nx, st.ny, st.gamma, st.mu, st.Pr, st.order, st.recon, st.bc_x,
                      st.bc_y, st.x0, st.x1, st.y0, st.y1, wall_T=st.wall_T,
                      wall_u=st.wall_u, **kw)
    O.set_state(st.W, st.Wx, st.Wy)
    return O


def _run(st, t_end, cfl=0.3, **kw):
    O = _solver(st, **kw)
    dt = cfl / O.max_wavespeed()
    n = math.ceil(t_end / dt)
    for _ in range(n):
        O.step(t_end / n)
    return O.get_state()


# ---- 1. the ghost map and its derivatives -----------------------------------------------
GAMMA = 1.4
WALL_T = (0.55, 0.65, 0.75, 0.85)   # distinct per wall: a wrong wall index shows
WALL_U = (0.11, -0.13, 0.17, -0.19)


def _prim_field(s, dim):
    """A smooth primitive field (rho, u, v, p) along a coordinate s."""
    rho = 1.0 + 0.3 * np.sin(1.3 * s + 0.2)
    u = 0.4 * np.cos(0.7 * s) - 0.1
    v = 0.25 * np.sin(0.9 * s + 0.5)
    p = 0.8 + 0.2 * np.cos(1.1 * s - 0.3)
    return (rho, u, v, p) if dim == 2 else (rho, u, p)


def _cons(prim, dim):
    if dim == 2:
        rho, u, v, p = prim
        return np.array([rho, rho * u, rho * v, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)])
    rho, u, p = prim
    return np.array([rho, rho * u, p / (GAMMA - 1) + 0.5 * rho * u * u])


def _ghost_prim(prim, dim, axis, side):
    """The ghost's primitive state by the wall map of R25 (the definition)."""
    k = 2 * (axis - 1) + side
    Tw, uw = WALL_T[k], WALL_U[k]
    if dim == 2:
        rho, u, v, p = prim
        vel = [u, v]
    else:
        rho, u, p = prim
        vel = [u]
    T = p / rho
    n = axis - 1
    g = [None] * dim
    g[n] = -vel[n]
    if dim == 2:
        g[1 - n] = 2 * uw - vel[1 - n]
    Tg = 2 * Tw - T
    return ((p / Tg, *g, p))


@pytest.mark.parametrize("dim,axis", [(1, 1), (2, 1), (2, 2)])
@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("normal", [True, False])
def test_iso_ghost_is_the_ghost_field(dim, axis, side, normal):
    if dim == 1 and not normal:
        pytest.skip("1D has no direction along the wall")
    O = oracle.Solver(8, 8 if dim == 2 else 1, GAMMA, 0.01, 0.72, 8, 0, 3, 3 if dim == 2 else 0,
                      wall_T=WALL_T, wall_u=WALL_U)
    h = 1e-5
    for s in (0.3, 1.7, -0.9):
        q = _cons(_prim_field(s, dim), dim)
        dq = (_cons(_prim_field(s + h, dim), dim) - _cons(_prim_field(s - h, dim), dim)) / (2 * h)
        wg, dg = O.iso_ghost(axis, side, normal, q, dq)
        G = lambda t: _cons(_ghost_prim(_prim_field(t, dim), dim, axis, side), dim)
        np.testing.assert_allclose(wg, G(s), rtol=1e-14, atol=1e-14)
        # across the wall the ghost at distance d outside mirrors the cell at d inside, so a
        # step outwards is a step inwards in the cell's coordinate
        fd = (G(s + h) - G(s - h)) / (2 * h)
        if normal:
            fd = -fd
        np.testing.assert_allclose(dg, fd, rtol=1e-8, atol=1e-8)


# ---- 2. plane Couette flow ---------------------------------------------------------------
def _couette_errors(st, W):
    """Max errors of u (relative to U) and T (relative to the peak heating) of the
    row-averaged solution, walls normal to y."""
    U, T0 = st.meta["U"], st.meta["T0"]
    yc = (np.arange(st.ny) + 0.5) / st.ny
    rho = W[0].mean(axis=1)
    u = W[1].mean(axis=1) / rho
    p = (st.gamma - 1) * (W[3].mean(axis=1) - 0.5 * W[1].mean(axis=1) ** 2 / rho)
    ue, Te = inputs.couette_profile(yc, U, T0, st.Pr, st.gamma)
    rise = st.Pr * U * U / (8 * st.gamma / (st.gamma - 1))
    return np.abs(u - ue).max() / U, np.abs(p / rho - Te).max() / rise


def test_couette_flow_second_order():
    errs = []
    for ny in (8, 16):
        st = inputs.couette_2d(ny)
        W = _run(st, 5.0)[0]
        assert np.abs(W[2]).max() < 1e-7 * W[0].max()   # acoustic transients only
        errs.append(_couette_errors(st, W))
    (u8, T8), (u16, T16) = errs
    assert u8 < 1e-6 and u16 < 2e-7, errs
    assert T16 < 3e-3 and T8 / T16 > 3.5, errs


def test_couette_flow_turned_walls_match():
    sy = inputs.couette_2d(8, nx=5, walls="y")
    sx = inputs.couette_2d(8, nx=5, walls="x")
    # same data turned: (x, y) -> (y, x), momenta swapped
    tr = lambda A: np.ascontiguousarray(np.swapaxes(A, 1, 2)[[0, 2, 1, 3]])
    np.testing.assert_allclose(sx.W, tr(sy.W), rtol=1e-15, atol=1e-15)
    Wy = _run(sy, 0.5)
    Wx = _run(sx, 0.5)
    for A, B in ((Wx[0], tr(Wy[0])), (Wx[1], tr(Wy[2])), (Wx[2], tr(Wy[1]))):
        np.testing.assert_allclose(A, B, rtol=0, atol=1e-12 * np.abs(B).max())


# ---- 3. heat conduction --------------------------------------------------------------------
def test_heat_conduction_second_order():
    errs = []
    for n in (8, 16):
        st = inputs.heat_conduction_1d(n)
        W = _run(st, 5.0)[0][:, 0, :]
        TL, TR = st.meta["TL"], st.meta["TR"]
        xc = (np.arange(n) + 0.5) / n
        T = (st.gamma - 1) * (W[2] - 0.5 * W[1] ** 2 / W[0]) / W[0]
        errs.append(np.abs(T - (TL + (TR - TL) * xc)).max() / (TR - TL))
        assert np.abs(W[1]).max() < 1e-5
    assert errs[1] < 3e-5 and errs[0] / errs[1] > 3.5, errs


# ---- 4. the cavity's mirror symmetry --------------------------------------------------------
@pytest.mark.parametrize("recon,order", [(0, 6), (1, 8)])
def test_cavity_lid_reversal_is_the_mirror_image(recon, order):
    st = inputs.lid_cavity_2d(10, order=order, recon=recon)
    st.mu = 0.01   # a coarse grid: keep the cell Reynolds number moderate
    U = st.meta["U"]
    a = _solver(st)
    rev = inputs.lid_cavity_2d(10, order=order, recon=recon)
    rev.mu = st.mu
    rev.wall_u = (0.0, 0.0, 0.0, -U)
    b = _solver(rev)
    dt = 0.3 / a.max_wavespeed()
    for _ in range(12):
        a.step(dt)
        b.step(dt)
    Wa, Wxa, Wya = a.get_state()
    Wb, Wxb, Wyb = b.get_state()
    s = np.array([1.0, -1.0, 1.0, 1.0]).reshape(4, 1, 1)
    mir = lambda A: np.flip(A, axis=2) * s
    tol = 1e-12 * np.abs(Wa).max()
    assert np.abs(Wa[1]).max() > 1e-3   # the lid has set the gas moving
    np.testing.assert_allclose(Wb, mir(Wa), rtol=0, atol=tol)
    np.testing.assert_allclose(Wyb, mir(Wya), rtol=0, atol=tol / st.dy)
    np.testing.assert_allclose(Wxb, -mir(Wxa), rtol=0, atol=tol / st.dx)


def test_gas_at_rest_at_the_wall_temperature_stays_at_rest():
    st = inputs.lid_cavity_2d(8, recon=1)
    st.wall_u = (0.0, 0.0, 0.0, 0.0)
    W0 = st.W.copy()
    W = _run(st, 0.3)[0]
    np.testing.assert_allclose(W, W0, rtol=0, atol=1e-13)


def test_moving_isothermal_wall_meeting_a_reflecting_wall_is_rejected():
    with pytest.raises(ValueError):
        oracle.Solver(8, 8, bc_x=2, bc_y=3, wall_u=(0.0, 0.0, 0.0, 0.1))
    oracle.Solver(8, 8, bc_x=2, bc_y=3, wall_u=(0.1, 0.0, 0.0, 0.0))   # the x walls' speeds are unused
