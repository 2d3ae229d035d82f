"""Isothermal no-slip walls (bc 3) on the GPU (FP64 form, through the C ABI): parity with the
oracle after one and two steps, and over a longer lid-driven cavity run.

Tolerance: that of the periodic parity tests (reading R22), 1e-12 per variable relative to
max |W|, slopes relative to max(max |W'|, max |W|/h); a momentum whose flow is (nearly) at
rest -- the normal momentum of Couette flow, both of heat conduction -- is measured against
the momentum scale rho c of the pressure that its flux carries (as the shear-wave parity test
measures its y momentum against the flow's).  Both sides build the rows of faces beyond a
wall from ghost cells, so the only differences are rounding in the ghost map.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1901_00261_gb300 import gks, inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gks.lib()


def rel_err(a, b, floor=None):
    worst = 0.0
    for v in range(b.shape[0]):
        scale = max(np.abs(b[v]).max(), 1e-300)
        if floor is not None:
            scale = max(scale, floor[v])
        worst = max(worst, np.abs(a[v] - b[v]).max() / scale)
    return worst


def oracle_of(st):
    O = oracle.Solver(st.nx, st.ny, st.gamma, st.mu, st.Pr, st.order, st.recon, st.bc_x,
                      st.bc_y, st.x0, st.x1, st.y0, st.y1, wall_T=st.wall_T, wall_u=st.wall_u)
    O.set_state(st.W, st.Wx, st.Wy)
    return O


def random_box(nx, ny, seed, order, recon, bc_x=3, bc_y=3):
    """2D data with no symmetry, between isothermal walls of four different temperatures and
    velocities: density and pressure in [0.9, 1.1], velocities in [-0.1, 0.1], slopes of the
    size of the cell-to-cell differences (wider jumps take the 2D linear scheme to
    non-physical states).  The viscosity 0.05 dx keeps mu dt / dx^2 near 0.01, well inside
    the explicit scheme's viscous limit."""
    mu = 0.05 / nx
    u = inputs.uniform01_array(seed, 12 * nx * ny).reshape(12, ny, nx)
    W = inputs.conservative_2d(0.9 + 0.2 * u[0], 0.2 * u[1] - 0.1, 0.2 * u[2] - 0.1,
                               0.9 + 0.2 * u[3], 1.4)
    Wx = (2.0 * u[4:8] - 1.0) * 0.02 * nx
    Wy = (2.0 * u[8:12] - 1.0) * 0.02 * ny
    return inputs.State(W, Wx, Wy, nx, ny, 1.4, 0.0, 1.0, 0.0, ny / nx, bc_x, bc_y, mu=mu,
                        Pr=0.72, order=order, recon=recon, name="random_box",
                        wall_T=(0.95, 1.05, 0.9, 1.1),
                        wall_u=(0.05 * (bc_y != 2), -0.06 * (bc_y != 2), 0.07 * (bc_x != 2),
                                -0.08 * (bc_x != 2)))


def random_tube(N, seed, order, recon):
    mu = 0.05 / N
    u = inputs.uniform01_array(seed, 6 * N).reshape(6, N)
    W = inputs.conservative_1d(0.8 + 0.4 * u[0], 0.4 * u[1] - 0.2, 0.8 + 0.4 * u[2], 1.4)
    Wx = (2.0 * u[3:6] - 1.0) * 0.05 * N
    return inputs.State(W.reshape(3, 1, N), Wx.reshape(3, 1, N), None, N, 1, 1.4, 0.0, 1.0,
                        bc_x=3, mu=mu, Pr=0.72, order=order, recon=recon, name="random_tube",
                        wall_T=(0.9, 1.1, 1.0, 1.0))


def compare(st, nsteps, tolw=TOL, tols=TOL):
    G = gks.Solver.from_state(st)
    O = oracle_of(st)
    dt = 0.3 / O.max_wavespeed()
    for _ in range(nsteps):
        G.step(dt)
        O.step(dt)
    g, o = G.get_state(), O.get_state()
    W = o[0]
    nv = W.shape[0]
    kin = sum(W[1 + d] ** 2 for d in range(nv - 2)) / W[0]
    p = (st.gamma - 1) * (W[nv - 1] - 0.5 * kin)
    rc = np.sqrt(st.gamma * p * W[0]).max()   # rho c
    floor_w = [0.0] + [rc] * (nv - 2) + [0.0]
    e = rel_err(g[0], o[0], floor_w)
    assert e <= tolw, f"{st.name} W: {e:.3e}"
    for k, h in ((1, st.dx), (2, st.dy)):
        if o[k] is not None:
            fl = [max(np.abs(W[v]).max(), floor_w[v]) / h for v in range(nv)]
            e = rel_err(g[k], o[k], fl)
            assert e <= tols, f"{st.name} slopes {k}: {e:.3e}"


CASES = [
    ("1D linear 6th, random, N=37", lambda: random_tube(37, 11, 6, 0), 2),
    ("1D WENO-Z 8th, random, N=300", lambda: random_tube(300, 12, 8, 1), 2),
    ("1D heat conduction 8th, N=40", lambda: inputs.heat_conduction_1d(40), 2),
    ("2D linear 8th, random, four walls, 37x29", lambda: random_box(37, 29, 13, 8, 0), 2),
    ("2D linear 6th, random, four walls, 5x5", lambda: random_box(5, 5, 14, 6, 0), 1),
    ("2D WENO-Z 8th, random, four walls, 40x36", lambda: random_box(40, 36, 15, 8, 1), 1),
    ("2D WENO-Z 6th, random, x walls, periodic y", lambda: random_box(33, 27, 16, 6, 1, bc_y=0), 2),
    ("2D linear 8th, random, reflecting x, isothermal y", lambda: random_box(30, 35, 17, 8, 0, bc_x=2), 2),
    ("2D linear 8th, transmissive x, isothermal y", lambda: random_box(31, 26, 18, 8, 0, bc_x=1), 2),
    ("2D Couette, walls y, 5x16", lambda: inputs.couette_2d(16), 2),
    ("2D Couette, walls x, 16x5", lambda: inputs.couette_2d(16, walls="x"), 2),
    ("2D cavity Re 1000, WENO-Z 8th, 33x33", lambda: inputs.lid_cavity_2d(33), 2),
]


@pytest.mark.parametrize("name,make,nsteps", CASES, ids=[c[0] for c in CASES])
def test_isothermal_walls_fp64_parity(name, make, nsteps):
    compare(make(), nsteps)


def test_cavity_forty_steps_parity():
    """The lid-driven cavity of Sec. 5 (Re 1000, lid speed 0.15, 8th-order WENO-Z) over 40
    steps from rest: rounding differences stay at the per-step level."""
    st = inputs.lid_cavity_2d(24)
    compare(st, 40, 1e-11, 1e-11)


def test_isothermal_walls_rejected_by_fp32_bulk():
    with pytest.raises(gks.GksError):
        gks.Solver(16, 16, bc_x=3, bc_y=3, precision=gks.PREC_FP32_BULK)
    with pytest.raises(gks.GksError):   # a moving isothermal wall meeting a reflecting one
        gks.Solver(16, 16, bc_x=2, bc_y=3, wall_u=(0.0, 0.0, 0.0, 0.1))


def test_couette_flow_on_the_gpu():
    """Couette flow at 64 rows (the oracle's pin runs 8 and 16; mu 0.002 keeps mu dt / dy^2
    at 0.03): the GPU keeps the closed-form profile within the second-order error that the
    oracle's rows extrapolate to."""
    st = inputs.couette_2d(64, mu=0.002)
    G = gks.Solver.from_state(st)
    dt0 = 0.3 / G.max_wavespeed()
    n = math.ceil(2.0 / dt0)
    for _ in range(n):
        G.step(2.0 / n)
    W = G.get_state()[0]
    U, T0 = st.meta["U"], st.meta["T0"]
    yc = (np.arange(st.ny) + 0.5) / st.ny
    rho = W[0].mean(axis=1)
    u = W[1].mean(axis=1) / rho
    T = 0.4 * (W[3].mean(axis=1) - 0.5 * W[1].mean(axis=1) ** 2 / rho) / rho
    ue, Te = inputs.couette_profile(yc, U, T0, st.Pr, st.gamma)
    rise = st.Pr * U * U / (8 * 3.5)
    assert np.abs(u - ue).max() / U < 2e-7
    assert np.abs(T - Te).max() / rise < 3e-4
