"""The tangential WENO-Z option (tan_mode = 1; the variant of the tangential reconstruction of
Sec. 3.1, last paragraph, that carries the WENO-Z of Sec. 3.3 across the face for the initial
non-equilibrium states) on the GPU, through the C ABI, against the oracle in the same mode.

FP64 form: one step from identical input within 1e-12 (the parity bound of
tests/test_gpu_parity.py).  FP32-bulk form: one step within its bounds against the FP64 form.
A y-independent Sod tube run as a 2D problem: with the option the library stays physical and
reproduces the 1D run in every row (the default reading goes non-physical on the y faces).
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


def rel(a, b, floor=None):
    """max over variables of max|a - b| / scale; a variable that vanishes in the data (V of a
    y-independent tube, rounding noise of ~1e-17 on either side) is measured against the
    largest variable's scale."""
    worst = 0.0
    big = max(np.abs(b[v]).max() for v in range(b.shape[0]))
    for v in range(b.shape[0]):
        scale = np.abs(b[v]).max()
        if scale < 1e-8 * big:
            scale = big
        scale = max(scale, 1e-300)
        if floor is not None:
            scale = max(scale, floor[v])
        worst = max(worst, np.abs(a[v] - b[v]).max() / scale)
    return worst


def sod_rows(N, ny, order):
    st = inputs.sod_1d(N, order=order, recon=1)
    W2, Wx2 = np.zeros((4, ny, N)), np.zeros((4, ny, N))
    for a, b in ((0, 0), (1, 1), (2, 3)):
        W2[b] = st.W[a, 0]
        Wx2[b] = st.Wx[a, 0]
    dy = (st.x1 - st.x0) / N
    return inputs.State(W2, Wx2, np.zeros_like(W2), N, ny, st.gamma, st.x0, st.x1, 0.0, ny * dy, 1, 0,
                        order=order, recon=1, name="sod_rows"), st


def oracle_of(st, tan_mode):
    O = oracle.Solver(st.nx, st.ny, st.gamma, st.mu, st.Pr, st.order, st.recon, st.bc_x, st.bc_y,
                      st.x0, st.x1, st.y0, st.y1, tan_mode=tan_mode)
    O.set_state(st.W, st.Wx, st.Wy)
    return O


CASES = [
    ("WENO-Z vortex 8th 40x33", lambda: inputs.isentropic_vortex_2d(40, order=8, recon=1, ny=33)),
    ("WENO-Z vortex 6th 37x29", lambda: inputs.isentropic_vortex_2d(37, order=6, recon=1, ny=29)),
    ("NS WENO-Z shear layer 48^2", lambda: inputs.shear_layer_2d(48)),
    ("grid-aligned Sod tube 8th 70x9", lambda: sod_rows(70, 9, 8)[0]),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_fp64_parity_with_tangential_weno(name, make):
    st = make()
    O = oracle_of(st, 1)
    G = gks.Solver.from_state(st, tan_mode=1)
    dt = 0.3 / O.max_wavespeed()
    for step in range(2):
        O.step(dt)
        G.step(dt)
        g, o = G.get_state(), O.get_state()
        assert rel(g[0], o[0]) <= TOL, f"{name} step {step} W"
        for k, h in ((1, st.dx), (2, st.dy)):
            fl = [np.abs(o[0][v]).max() / h for v in range(4)]
            assert rel(g[k], o[k], fl) <= TOL, f"{name} step {step} slopes {k}"


@pytest.mark.parametrize("name,make,tolw,tols", [
    ("WENO-Z vortex 8th 64^2", lambda: inputs.isentropic_vortex_2d(64, order=8, recon=1), 3e-7, 2e-6),
    ("NS WENO-Z shear layer 64^2", lambda: inputs.shear_layer_2d(64), 2e-5, 2e-5),
    ("grid-aligned Sod tube 8th 200x8", lambda: sod_rows(200, 8, 8)[0], 2e-6, 2e-6)])
def test_fp32_bulk_with_tangential_weno_close_to_fp64(name, make, tolw, tols):
    st = make()
    A = gks.Solver.from_state(st, precision=gks.PREC_FP32_BULK, tan_mode=1)
    B = gks.Solver.from_state(st, precision=gks.PREC_FP64, tan_mode=1)
    dt = 0.3 / B.max_wavespeed()
    A.step(dt)
    B.step(dt)
    a, b = A.get_state(), B.get_state()
    assert rel(a[0], b[0]) <= tolw
    for k, h in ((1, st.dx), (2, st.dy)):
        assert rel(a[k], b[k], [np.abs(b[0][v]).max() / h for v in range(4)]) <= tols


@pytest.mark.parametrize("prec", [gks.PREC_FP64, gks.PREC_FP32_BULK])
def test_grid_aligned_sod_tube_equals_the_1d_run(prec):
    """30 steps of the y-independent Sod tube in 2D with the option: every row equals the
    library's own 1D run (FP64: 1e-11 of max|W|; FP32-bulk: its single-precision rounding,
    1e-5); without the option the first step reports a non-physical state."""
    st2, st1 = sod_rows(160, 6, 8)
    G2 = gks.Solver.from_state(st2, precision=prec, tan_mode=1)
    G1 = gks.Solver.from_state(st1, precision=prec)
    dt = 0.3 / G1.max_wavespeed()
    G2.steps(dt, 30)
    G1.steps(dt, 30)
    a, _, _ = G1.get_state()
    b, _, by = G2.get_state()
    tol = 1e-11 if prec == gks.PREC_FP64 else 1e-5
    for ia, ib in ((0, 0), (1, 1), (2, 3)):
        assert np.abs(b[ib] - a[ia]).max() <= tol * np.abs(a[ia]).max(), (ia, ib)
    G0 = gks.Solver.from_state(st2, precision=prec)
    G0.step(dt)
    with pytest.raises(gks.GksError) as ei:
        G0.get_state()
    assert ei.value.code == gks.GKS_ENONPHYSICAL
