"""Reflecting walls on the GPU (through the C ABI): parity with the oracle in both forms and
the mirror symmetry at a size the oracle does not run.

Tolerances are those of the periodic parity tests: 1e-12 for the FP64 form after one or two
steps (per variable, relative to max |W|; slopes relative to max(max |W'|, max |W|/h)), the
FP32-bulk bounds of its comparison with FP64.  The Navier-Stokes WENO-Z case compares after
one step: beyond a wall the GPU reconstructs mirrored cells while the oracle mirrors the
reconstructed face row, which agree to rounding of the characteristic projection; WENO-Z
weights of nearly constant characteristic fields react to that rounding, and the viscous
second derivatives carry it to ~1e-12 of the slopes after a second step.
"""
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
                      st.bc_y, st.x0, st.x1, st.y0, st.y1)
    O.set_state(st.W, st.Wx, st.Wy)
    return O


def random_tube(N, seed, order, recon):
    """1D data with no symmetry between walls: density and pressure in [0.8, 1.2],
    velocity in [-0.4, 0.4], slopes of the size of the cell-to-cell differences."""
    u = inputs.uniform01_array(seed, 6 * N).reshape(6, N)
    W = inputs.conservative_1d(0.8 + 0.4 * u[0], 0.8 * u[1] - 0.4, 0.8 + 0.4 * u[2], 1.4)
    Wx = (2.0 * u[3:6] - 1.0) * 0.05 * N
    return inputs.State(W.reshape(3, 1, N), Wx.reshape(3, 1, N), None, N, 1, 1.4, 0.0, 1.0,
                        bc_x=2, order=order, recon=recon, name="random_tube")


def compare(st, nsteps, precision, tolw, tols):
    G = gks.Solver.from_state(st, precision=precision)
    O = oracle_of(st)
    dt = 0.3 / O.max_wavespeed()
    for _ in range(nsteps):
        G.step(dt)
        O.step(dt)
    g, o = G.get_state(), O.get_state()
    e = rel_err(g[0], o[0])
    assert e <= tolw, f"{st.name} W: {e:.3e}"
    for k, h in ((1, st.dx), (2, st.dy)):
        if o[k] is not None:
            e = rel_err(g[k], o[k], [np.abs(o[0][v]).max() / h for v in range(o[0].shape[0])])
            assert e <= tols, f"{st.name} slopes {k}: {e:.3e}"


FP64_CASES = [
    ("1D linear 6th, N=37", lambda: random_tube(37, 1, 6, 0), 2),
    ("1D linear 8th, N=1000", lambda: random_tube(1000, 2, 8, 0), 2),
    ("1D WENO-Z 8th, N=300", lambda: random_tube(300, 3, 8, 1), 2),
    ("1D WENO-Z 6th wall impact, N=400", lambda: inputs.wall_impact_1d(400, order=6), 2),
    ("2D linear 8th, walls x and y, 37x29", lambda: inputs.box_pulse_2d(37, ny=29), 2),
    ("2D linear 8th, walls x and y, 5x5", lambda: inputs.box_pulse_2d(5, ny=5), 1),
    ("2D WENO-Z 6th, walls x and y, 40x36", lambda: inputs.box_pulse_2d(40, ny=36, order=6, recon=1), 2),
    ("2D linear 6th, walls x, periodic y", lambda: inputs.box_pulse_2d(33, ny=27, order=6, bc_y=0), 2),
    ("2D WENO-Z 8th, transmissive x, walls y", lambda: inputs.box_pulse_2d(30, ny=35, recon=1, bc_x=1), 2),
    ("2D NS WENO-Z 8th, walls x and y", lambda: inputs.box_pulse_2d(32, ny=28, recon=1, mu=2e-3, Pr=0.72), 1),
]


@pytest.mark.parametrize("name,make,nsteps", FP64_CASES, ids=[c[0] for c in FP64_CASES])
def test_walls_fp64_parity(name, make, nsteps):
    compare(make(), nsteps, gks.PREC_FP64, TOL, TOL)


# FP32-bulk form: the bounds of its comparison with FP64 on the periodic workloads (smooth
# data); the random tube's 20 % cell-to-cell jumps, and the box pulse under WENO-Z (about
# nine cells across its width, where the WENO-Z weights react to single-precision rounding:
# 5.7e-7 measured), take the bound of the 1D WENO-Z cases
FP32_CASES = [
    ("1D WENO-Z 8th wall impact, N=1000", lambda: inputs.wall_impact_1d(1000), 2e-6, 2e-6),
    ("1D linear 8th, N=1000", lambda: random_tube(1000, 4, 8, 0), 2e-6, 2e-6),
    ("2D linear 8th, walls x and y, 64x48", lambda: inputs.box_pulse_2d(64, ny=48), 3e-8, 3e-7),
    ("2D WENO-Z 8th, walls x and y, 64x64", lambda: inputs.box_pulse_2d(64, recon=1), 2e-6, 2e-6),
    ("2D NS WENO-Z 8th, walls y, 48x40", lambda: inputs.box_pulse_2d(48, ny=40, recon=1, mu=2e-3, Pr=0.72, bc_x=0), 2e-5, 2e-5),
]


@pytest.mark.parametrize("name,make,tolw,tols", FP32_CASES, ids=[c[0] for c in FP32_CASES])
def test_walls_fp32_bulk_close_to_oracle(name, make, tolw, tols):
    compare(make(), 1, gks.PREC_FP32_BULK, tolw, tols)


def test_walls_conserve_mass_and_energy_fp32_bulk():
    st = inputs.box_pulse_2d(96, ny=80, recon=1)
    S = gks.Solver.from_state(st, precision=gks.PREC_FP32_BULK)
    W0 = S.get_state()[0]
    S.steps(0.3 / S.max_wavespeed(), 10)
    W = S.get_state()[0]
    for v in (0, 3):
        assert abs(W[v].sum() - W0[v].sum()) <= 1e-13 * np.abs(W0[v]).sum()


def _mirror_extend(st):
    """The periodic problem on [0, 2]^2 equivalent to st between walls on [0, 1]^2."""
    def flip(W, Wn, Wt, var, axis):
        s = np.ones((4, 1, 1))
        s[var] = -1.0
        return (np.flip(W, axis) * s, np.flip(Wn, axis) * -s, np.flip(Wt, axis) * s)
    Wm, Wxm, Wym = flip(st.W, st.Wx, st.Wy, 1, 2)
    W = np.concatenate([st.W, Wm], 2)
    Wx = np.concatenate([st.Wx, Wxm], 2)
    Wy = np.concatenate([st.Wy, Wym], 2)
    Wm, Wym, Wxm = flip(W, Wy, Wx, 2, 1)
    W, Wx, Wy = (np.concatenate([W, Wm], 1), np.concatenate([Wx, Wxm], 1),
                 np.concatenate([Wy, Wym], 1))
    return inputs.State(np.ascontiguousarray(W), np.ascontiguousarray(Wx),
                        np.ascontiguousarray(Wy), 2 * st.nx, 2 * st.ny, st.gamma, 0.0,
                        2.0 * st.x1, 0.0, 2.0 * st.y1, 0, 0, order=st.order, recon=st.recon)


# FP32-bulk: the wall run and the periodic run use different instantiations of the sweeps
# (with and without the wall signs), whose single-precision rounding may differ
@pytest.mark.parametrize("recon,precision,tolw,tols", [
    (0, gks.PREC_FP64, 1e-12, 1e-12), (1, gks.PREC_FP64, 1e-12, 1e-12),
    (0, gks.PREC_FP32_BULK, 1e-7, 1e-6), (1, gks.PREC_FP32_BULK, 1e-6, 1e-5)],
    ids=["fp64 linear", "fp64 weno", "fp32 linear", "fp32 weno"])
def test_walls_equal_mirrored_periodic_at_512(recon, precision, tolw, tols):
    # 512^2 between walls against 1024^2 periodic: many tiles, both forms of the ghost
    # rows (normal and tangential), at a size the oracle does not run
    st = inputs.box_pulse_2d(512, recon=recon)
    ext = _mirror_extend(st)
    A = gks.Solver.from_state(st, precision=precision)
    B = gks.Solver.from_state(ext, precision=precision)
    dt = 0.3 / A.max_wavespeed()
    A.steps(dt, 2)
    B.steps(dt, 2)
    a, b = A.get_state(), B.get_state()
    n = st.nx
    assert rel_err(a[0], b[0][:, :n, :n]) <= tolw
    fl = [np.abs(b[0][v]).max() / st.dx for v in range(4)]
    assert rel_err(a[1], b[1][:, :n, :n], fl) <= tols
    assert rel_err(a[2], b[2][:, :n, :n], fl) <= tols
