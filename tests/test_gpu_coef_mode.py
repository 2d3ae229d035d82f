"""The full-product variant of the equilibrium Taylor coefficients (reading R6, gks_opts.coef_mode
= 1) on the GPU (FP64 form, through the C ABI): parity with the oracle's variant after one
and two steps, 1e-12 per variable as the default reading's parity tests (reading R22).  The
kernels add the Euler fluxes' second derivatives to the linearised chain (closed forms); the
oracle keeps the Maxwellian's Taylor products in its moment integrals: two routes to the same
interface values."""
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


def compare(st, nsteps):
    G = gks.Solver.from_state(st, coef_mode=1)
    O = oracle.Solver(st.nx, st.ny, st.gamma, st.mu, st.Pr, st.order, st.recon, st.bc_x,
                      st.bc_y, st.x0, st.x1, st.y0, st.y1, coef_mode=1)
    O.set_state(st.W, st.Wx, st.Wy)
    dt = 0.3 / O.max_wavespeed()
    for _ in range(nsteps):
        G.step(dt)
        O.step(dt)
    g, o = G.get_state(), O.get_state()
    assert rel_err(g[0], o[0]) <= TOL, st.name
    for k, h in ((1, st.dx), (2, st.dy)):
        if o[k] is not None:
            fl = [np.abs(o[0][v]).max() / h for v in range(o[0].shape[0])]
            assert rel_err(g[k], o[k], fl) <= TOL, (st.name, k)
    # the variant is not the default reading
    D = gks.Solver.from_state(st)
    for _ in range(nsteps):
        D.step(dt)
    return rel_err(D.get_state()[1], g[1])


CASES = [
    ("1D linear 6th, density wave, N=37", lambda: inputs.density_wave_1d(37, order=6, recon=0), 2),
    ("1D WENO-Z 8th, Sod, N=200", lambda: inputs.sod_1d(200, order=8, recon=1), 2),
    ("2D linear 8th, vortex, 37x29", lambda: inputs.isentropic_vortex_2d(37, order=8, recon=0, ny=29), 2),
    ("2D linear 6th, vortex, 5x5", lambda: inputs.isentropic_vortex_2d(5, order=6, recon=0), 1),
    ("2D WENO-Z 8th, vortex, 40x36", lambda: inputs.isentropic_vortex_2d(40, order=8, recon=1, ny=36), 2),
    ("2D linear 8th, walls, 33x27", lambda: inputs.box_pulse_2d(33, ny=27), 2),
]


@pytest.mark.parametrize("name,make,nsteps", CASES, ids=[c[0] for c in CASES])
def test_full_product_coefficients_parity(name, make, nsteps):
    diff = compare(make(), nsteps)
    if "vortex" in name:
        assert diff > 1e-9   # the slopes of a nonlinear flow see the product terms


def test_full_product_coefficients_rejected_where_undefined():
    with pytest.raises(gks.GksError):
        gks.Solver(16, 16, coef_mode=1, precision=gks.PREC_FP32_BULK)
    with pytest.raises(gks.GksError):
        gks.Solver(16, 16, mu=0.01, coef_mode=1)
    with pytest.raises(gks.GksError):
        gks.Solver(16, 16, tau_mode=1, coef_mode=1)
