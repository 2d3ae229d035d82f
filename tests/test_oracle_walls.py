"""Pins of the oracle's reflecting walls (reading R24: a ghost cell is the mirror image of
the cell at the same distance inside; the wall-normal momentum changes sign, and so do the
wall-normal derivatives of the other variables).

1. Symmetry: a solution on [0, 1] between walls is, cell for cell, the solution on the
   periodic [0, 2] of the data extended by its mirror image about x = 1 (the extension is
   even about both x = 0 = 2 and x = 1, and the scheme keeps that symmetry).  This ties the
   wall treatment to the periodic path, which the accuracy pins already fix; a dropped sign
   on a ghost's momentum or slope, or a ghost taken from the wrong cell, breaks it.
2. Physics: a uniform flow towards the walls.  Before the two wave systems meet, the
   solution next to each wall is the exact Riemann problem of the state against its mirror
   image (two shocks at the wall the flow runs into, two rarefactions at the other).
3. Conservation: no mass or energy crosses a wall.
"""
import numpy as np
import pytest

import oracle
from paper_1901_00261_gb300 import inputs

from riemann_exact import cell_average_density


def _solver(st, **kw):
    O = oracle.Solver(st.nx, st.ny, st.gamma, st.mu, st.Pr, st.order, st.recon, st.bc_x,
                      st.bc_y, st.x0, st.x1, st.y0, st.y1, **kw)
    O.set_state(st.W, st.Wx, st.Wy)
    return O


def _mirror(W, Wn, Wt, axis_var, array_axis):
    """Mirror image of (W, normal slope Wn, tangential slope Wt) across a wall: reversed
    along array_axis; the momentum component axis_var flips, and the normal slopes carry an
    extra sign (derivative of a mirrored function)."""
    s = np.ones(W.shape[0])
    s[axis_var] = -1.0
    sh = (-1,) + (1,) * (W.ndim - 1)
    Wm = np.flip(W, axis=array_axis) * s.reshape(sh)
    Wnm = np.flip(Wn, axis=array_axis) * (-s).reshape(sh)
    Wtm = None if Wt is None else np.flip(Wt, axis=array_axis) * s.reshape(sh)
    return Wm, Wnm, Wtm


def _extend(st, along_x, along_y):
    """The periodic problem on the doubled domain equivalent to st between walls."""
    W, Wx, Wy = st.W, st.Wx, st.Wy
    if along_x:
        Wm, Wxm, Wym = _mirror(W, Wx, Wy, 1, 2)
        W, Wx = np.concatenate([W, Wm], axis=2), np.concatenate([Wx, Wxm], axis=2)
        if Wy is not None:
            Wy = np.concatenate([Wy, Wym], axis=2)
    if along_y:
        Wm, Wym, Wxm = _mirror(W, Wy, Wx, 2, 1)
        W, Wx, Wy = (np.concatenate([W, Wm], axis=1), np.concatenate([Wx, Wxm], axis=1),
                     np.concatenate([Wy, Wym], axis=1))
    ny = W.shape[1]
    nx = W.shape[2]
    x1 = st.x0 + 2 * (st.x1 - st.x0) if along_x else st.x1
    y1 = st.y0 + 2 * (st.y1 - st.y0) if along_y else st.y1
    ext = inputs.State(np.ascontiguousarray(W), np.ascontiguousarray(Wx),
                       None if Wy is None else np.ascontiguousarray(Wy), nx, ny, st.gamma,
                       st.x0, x1, st.y0, y1, 0 if along_x else st.bc_x,
                       0 if along_y else st.bc_y, mu=st.mu, Pr=st.Pr, order=st.order,
                       recon=st.recon)
    return ext


def _random_tube(N, seed, order, recon):
    """Cell data with no symmetry: positive density and pressure, velocities up to 0.4,
    slopes of the size of the cell-to-cell differences."""
    u = inputs.uniform01_array(seed, 6 * N).reshape(6, N)
    rho = 0.8 + 0.4 * u[0]
    vel = 0.8 * u[1] - 0.4
    p = 0.8 + 0.4 * u[2]
    W = inputs.conservative_1d(rho, vel, p, 1.4).reshape(3, 1, N)
    Wx = (2.0 * u[3:6] - 1.0).reshape(3, 1, N) * 0.05 * N
    return inputs.State(W, Wx, None, N, 1, 1.4, 0.0, 1.0, bc_x=2, order=order, recon=recon)


def _step_both(st, nsteps, **kw):
    A = _solver(st, **kw)
    ext = _extend(st, st.bc_x == 2, st.ny > 1 and st.bc_y == 2)
    B = _solver(ext, **kw)
    dt = 0.3 / A.max_wavespeed()
    for _ in range(nsteps):
        A.step(dt)
        B.step(dt)
    return A.get_state(), B.get_state(), st


def _close(a, b, floor, tol):
    for v in range(a.shape[0]):
        scale = max(np.abs(b[v]).max(), floor[v])
        err = np.abs(a[v] - b[v]).max() / scale
        assert err <= tol, (v, err)


@pytest.mark.parametrize("order,recon", [(6, 0), (8, 0), (8, 1), (6, 1)])
def test_walls_1d_equal_mirrored_periodic(order, recon):
    st = _random_tube(24, seed=11 + order + recon, order=order, recon=recon)
    (a, ax, _), (b, bx, _), _ = _step_both(st, 2)
    N = st.nx
    _close(a, b[:, :, :N], [0.0] * 3, 1e-12)
    _close(ax, bx[:, :, :N], [np.abs(b[v]).max() * N for v in range(3)], 1e-12)


# The two runs differ only in how the face rows beyond a wall are formed (the wall run
# mirrors the reconstructed row; the periodic run reconstructs mirrored cells), so they
# agree to rounding of the characteristic projection.  Where a characteristic field is
# nearly constant the WENO-Z smoothness indicators are themselves rounding-sized and
# react to it; with the viscous terms' second derivatives this reaches ~1e-12 of the
# slopes after a second step, hence one step for the Navier-Stokes case.
@pytest.mark.parametrize("recon,mu,bcy,nsteps", [(0, 0.0, 2, 2), (1, 0.0, 2, 2), (1, 2e-3, 2, 1),
                                                 (0, 0.0, 0, 2)])
def test_walls_2d_equal_mirrored_periodic(recon, mu, bcy, nsteps):
    st = inputs.box_pulse_2d(12, ny=10, recon=recon, mu=mu, Pr=0.72 if mu else 1.0, bc_y=bcy)
    (a, ax, ay), (b, bx, by), _ = _step_both(st, nsteps)
    ny, nx = st.ny, st.nx
    fl = [np.abs(b[v]).max() * max(nx, ny) / min(st.x1 - st.x0, st.y1 - st.y0) for v in range(4)]
    _close(a, b[:, :ny, :nx], [0.0] * 4, 1e-12)
    _close(ax, bx[:, :ny, :nx], fl, 1e-12)
    _close(ay, by[:, :ny, :nx], fl, 1e-12)


def test_wall_mirror_sign_is_needed():
    # Planted mistake on the input side: the same tube with its mirror extension built
    # without the momentum sign is a different problem, and the comparison sees it.
    st = _random_tube(24, seed=3, order=8, recon=0)
    A = _solver(st)
    ext = _extend(st, True, False)
    N = st.nx
    ext.W[1, :, N:] *= -1.0
    ext.Wx[1, :, N:] *= -1.0
    B = _solver(ext)
    dt = 0.3 / A.max_wavespeed()
    A.step(dt)
    B.step(dt)
    assert np.abs(A.get_state()[0] - B.get_state()[0][:, :, :N]).max() > 1e-6


@pytest.mark.parametrize("N", [200, 400])
def test_wall_impact_matches_exact_riemann(N):
    st = inputs.wall_impact_1d(N, u0=0.5)
    O = _solver(st)
    t, T = 0.0, st.t_end
    while t < T - 1e-14:
        dt = min(0.3 / O.max_wavespeed(), T - t)
        O.step(dt)
        t += dt
    rho = O.get_state()[0][0, 0]
    rho0, u0, p0 = st.meta["state"]
    # x > 1/2: (rho, u0, p) | (rho, -u0, p) about x = 1; x < 1/2: the mirror about x = 0
    right = cell_average_density(N, 0.0, 1.0, 1.0, T, (rho0, u0, p0), (rho0, -u0, p0))
    left = cell_average_density(N, 0.0, 1.0, 0.0, T, (rho0, -u0, p0), (rho0, u0, p0))
    exact = np.where(np.arange(N) < N // 2, left, right)
    l1 = np.abs(rho - exact).mean()
    # first-order convergence at the shocks: L1 ~ C / N with C of the jump size
    assert l1 < 2.0 / N, l1
    # the wall holds the gas at rest: the state next to the right wall is the shocked star
    # state, whose density the exact solver gives
    assert abs(rho[-3:].mean() - right[-3:].mean()) < 5e-3 * right[-1]


@pytest.mark.parametrize("make", [lambda: inputs.box_pulse_2d(16, ny=12, recon=1),
                                  lambda: inputs.wall_impact_1d(60)])
def test_walls_conserve_mass_and_energy(make):
    st = make()
    O = _solver(st)
    dt = 0.3 / O.max_wavespeed()
    W0 = O.get_state()[0]
    for _ in range(4):
        O.step(dt)
    W = O.get_state()[0]
    for v in (0, W.shape[0] - 1):
        assert abs(W[v].sum() - W0[v].sum()) <= 1e-13 * np.abs(W0[v]).sum()


def test_oracle_rejects_unknown_boundary():
    with pytest.raises(ValueError):
        oracle.Solver(10, 1, bc_x=4)
