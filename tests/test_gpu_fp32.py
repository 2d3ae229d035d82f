"""FP32-bulk form against the FP64 form (both through the C ABI) and against exact solutions.

The FP32-bulk form runs the face-sweep arithmetic in single precision on differences from a
reference cell and keeps the time coefficients and the MSMD accumulation in FP64.  Its
error is therefore set by single-precision rounding of those differences (about 1e-7 of
dx |grad W| per face), not by the scheme.  Bounds below: per step against the FP64 form
(slopes relative to the scale max|W|/dx of their difference quotient), exact conservation,
and accuracy against the exact solutions where FP32 rounding is not yet dominant.
"""
import math

import numpy as np
import pytest

from paper_1901_00261_gb300 import gks, inputs
import acoustic_exact
import riemann_exact

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gks.lib()


def rel(a, b, floor=None):
    worst = 0.0
    for v in range(b.shape[0]):
        scale = max(np.abs(b[v]).max(), 1e-300)
        if floor is not None:
            scale = max(scale, floor[v])
        worst = max(worst, np.abs(a[v] - b[v]).max() / scale)
    return worst


def fp32_vs_fp64(st, nsteps=1):
    A = gks.Solver.from_state(st, precision=gks.PREC_FP32_BULK)
    B = gks.Solver.from_state(st, precision=gks.PREC_FP64)
    dt = 0.3 / B.max_wavespeed()
    A.steps(dt, nsteps)
    B.steps(dt, nsteps)
    a, b = A.get_state(), B.get_state()
    errs = [rel(a[0], b[0])]
    for k, h in ((1, st.dx), (2, st.dy)):
        if b[k] is not None:
            errs.append(rel(a[k], b[k], [np.abs(b[0][v]).max() / h for v in range(b[0].shape[0])]))
    return errs, a, st


# (name, input, bound for W, bound for the slopes); the bounds are ~10x the differences
# measured on a GB300 (linear paths ~2e-10 / ~1e-8, WENO-Z ~1e-7, NS ~1e-6).
CASES = [
    ("linear 1D 6th N=80", lambda: inputs.density_wave_1d(80, order=6), 3e-9, 3e-8),
    ("linear 1D 8th N=1000", lambda: inputs.density_wave_1d(1000, order=8), 3e-9, 3e-8),
    ("linear 2D 8th 64^2", lambda: inputs.isentropic_vortex_2d(64, order=8), 3e-8, 3e-7),
    ("linear 2D 6th 37x29", lambda: inputs.isentropic_vortex_2d(37, order=6, ny=29), 3e-8, 3e-7),
    ("WENO-Z 1D Sod N=1000", lambda: inputs.sod_1d(1000), 2e-6, 2e-6),
    ("WENO-Z 1D Shu-Osher N=400", lambda: inputs.shu_osher_1d(400), 2e-6, 2e-6),
    ("WENO-Z 2D vortex 64^2", lambda: inputs.isentropic_vortex_2d(64, order=8, recon=1), 3e-7, 2e-6),
    ("NS WENO-Z shear layer 64^2", lambda: inputs.shear_layer_2d(64), 2e-5, 2e-5),
]


@pytest.mark.parametrize("name,make,tolw,tols", CASES, ids=[c[0] for c in CASES])
def test_fp32_bulk_one_step_close_to_fp64(name, make, tolw, tols):
    errs, _, _ = fp32_vs_fp64(make())
    assert errs[0] <= tolw, f"{name}: W {errs[0]:.3e}"
    assert max(errs[1:]) <= tols, f"{name}: slopes {errs[1:]}"


@pytest.mark.parametrize("make", [lambda: inputs.isentropic_vortex_2d(96, order=8),
                                  lambda: inputs.shear_layer_2d(64),
                                  lambda: inputs.density_wave_1d(200, order=8, recon=1)])
def test_fp32_bulk_conserves_exactly(make):
    st = make()
    A = gks.Solver.from_state(st, precision=gks.PREC_FP32_BULK)
    dt = 0.3 / A.max_wavespeed()
    A.steps(dt, 5)
    W, _, _ = A.get_state()
    m0 = st.W.sum(axis=(1, 2))
    assert np.abs(W.sum(axis=(1, 2)) - m0).max() <= 1e-13 * np.abs(st.W).sum(axis=(1, 2)).max()


def _vortex_l1(n, prec, T=1.0):
    st = inputs.isentropic_vortex_2d(n, order=8)
    S = gks.Solver.from_state(st, precision=prec)
    ns = math.ceil(T / (0.3 / S.max_wavespeed()))
    S.steps(T / ns, ns)
    W, _, _ = S.get_state()
    return np.abs(W[0] - inputs.vortex_exact_avg(n, T)[0]).mean()


@pytest.mark.parametrize("n", [128, 256])
def test_fp32_bulk_vortex_accuracy_within_2x_of_fp64(n):
    """Isentropic vortex, 8th order, t = 1: L1 density error of the FP32-bulk form within a
    factor 2 of the FP64 form.  The factor-2 claim holds up to 256^2 at t = 1; on finer grids
    the FP32 rounding floor (next test) is above the FP64 form's truncation error."""
    e64, e32 = _vortex_l1(n, gks.PREC_FP64), _vortex_l1(n, gks.PREC_FP32_BULK)
    assert e32 <= 2.0 * e64, (e32, e64)


def test_fp32_bulk_vortex_error_at_512_where_the_factor_2_fails():
    """The first grid where the factor 2 is NOT met, pinned at its measured value: at t = 1
    the FP32-bulk L1 density error is 2.77e-8 (GB300), the FP64 form's 5.34e-10, a ratio of
    52; bounded here by 5e-8.  The cause is the weakly unstable high-frequency mode of the 2D
    linear scheme (both forms, and the oracle), which grows from the rounding of each form:
    ~1e-8 in FP32-bulk, ~1e-16 in FP64 (at 1024^2, t = 1: 1.1e-4 against 2.9e-9)."""
    e64, e32 = _vortex_l1(512, gks.PREC_FP64), _vortex_l1(512, gks.PREC_FP32_BULK)
    assert e32 <= 5e-8 and e64 < 1e-9, (e32, e64)
    assert e32 > 2.0 * e64   # the documented limit of the factor-2 claim still stands


def test_fp32_bulk_density_wave_error_floor():
    """Table 1 configuration (6th-order linear, N = 80, t = 2): the FP64 form gives the
    printed 1.220e-10; the FP32-bulk form stays below 3e-9 (its rounding floor)."""
    N = 80
    st = inputs.density_wave_1d(N, order=6)
    S = gks.Solver.from_state(st, precision=gks.PREC_FP32_BULK)
    n = math.ceil(2.0 / (0.3 * (2.0 / N) ** 1.5))
    S.steps(2.0 / n, n)
    W, _, _ = S.get_state()
    L1 = np.abs(W[0, 0] - inputs.density_wave_exact_rho(N, 2.0)).mean()
    assert L1 < 3e-9


def test_fp32_bulk_acoustic_wave():
    """Sec. 4.3 acoustic wave, N = 40, 8th order, t = 0.01 (1389 steps): a 1e-5 perturbation on a
    101325 background, which single precision alone could not resolve.  With its differences
    from the reference cell in single precision the FP32-bulk form follows linear acoustics
    within 1e-3 of the perturbation amplitude, and within 1e-4 of the FP64 form's error."""
    T, N = 0.01, 40
    errs = {}
    for prec in (gks.PREC_FP64, gks.PREC_FP32_BULK):
        st = inputs.acoustic_1d(N, order=8, recon=0)
        S = gks.Solver.from_state(st, precision=prec)
        n = math.ceil(T / (0.3 / S.max_wavespeed()))
        S.steps(T / n, n)
        W, _, _ = S.get_state()
        errs[prec] = np.abs(W[0, 0] - acoustic_exact.cell_average_density(N, T)).max() / acoustic_exact.amplitude()
    assert errs[gks.PREC_FP32_BULK] < 1e-3, errs
    assert abs(errs[gks.PREC_FP32_BULK] - errs[gks.PREC_FP64]) < 1e-4, errs


def _run_to(st, T, prec):
    S = gks.Solver.from_state(st, precision=prec)
    n = math.ceil(T / (0.3 / S.max_wavespeed()))
    S.steps(T / n, n)
    W, _, _ = S.get_state()
    S.close()
    return W


def test_fp32_bulk_shu_osher_against_fine_reference():
    """Shu-Osher (8th-order WENO-Z, N = 400, t = 1.8): L1 density error against a 12800-cell
    FP64 run averaged onto the 400 cells.  The FP32-bulk form's error is within 5 % of the FP64
    form's (the single-precision rounding is far below the discretisation error here)."""
    T, N, R = 1.8, 400, 32
    ref = _run_to(inputs.shu_osher_1d(N * R), T, gks.PREC_FP64)[0, 0].reshape(N, R).mean(axis=1)
    e = {p: np.abs(_run_to(inputs.shu_osher_1d(N), T, p)[0, 0] - ref).mean()
         for p in (gks.PREC_FP64, gks.PREC_FP32_BULK)}
    assert e[gks.PREC_FP64] < 0.05, e
    assert e[gks.PREC_FP32_BULK] <= 1.05 * e[gks.PREC_FP64], e


def test_fp32_bulk_sod_against_exact():
    """Sod tube (8th-order WENO-Z, N = 1000, t = 0.2): L1 density error against the exact
    Riemann solution's cell averages; the FP32-bulk form within 5 % of the FP64 form."""
    T, N = 0.2, 1000
    ex = riemann_exact.cell_average_density(N, 0.0, 1.0, 0.5, T, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    e = {p: np.abs(_run_to(inputs.sod_1d(N), T, p)[0, 0] - ex).mean()
         for p in (gks.PREC_FP64, gks.PREC_FP32_BULK)}
    assert e[gks.PREC_FP64] < 2e-3, e
    assert e[gks.PREC_FP32_BULK] <= 1.05 * e[gks.PREC_FP64], e


def test_fp32_bulk_full_size_vortex_step():
    """The benchmark configuration itself (2048^2, 8th order, linear, the same launches): one
    FP32-bulk step over the whole grid against the FP64 step within the 2D linear per-step bounds
    (W 3e-8, slopes 3e-7 of max|W|/h), and conservation to FP64 rounding."""
    st = inputs.isentropic_vortex_2d(2048, order=8)
    A = gks.Solver.from_state(st, precision=gks.PREC_FP32_BULK)
    dt = 0.3 / A.max_wavespeed()
    A.step(dt)
    a = A.get_state()
    A.close()
    B = gks.Solver.from_state(st, precision=gks.PREC_FP64)
    B.step(dt)
    b = B.get_state()
    B.close()
    assert rel(a[0], b[0]) <= 3e-8
    for k, h in ((1, st.dx), (2, st.dy)):
        assert rel(a[k], b[k], [np.abs(b[0][v]).max() / h for v in range(4)]) <= 3e-7
    m0 = st.W.sum(axis=(1, 2))
    assert np.abs(a[0].sum(axis=(1, 2)) - m0).max() <= 1e-12 * np.abs(st.W).sum(axis=(1, 2)).max()


def test_fp32_bulk_set_state_refreshes_mirror():
    st = inputs.isentropic_vortex_2d(48, order=8)
    A = gks.Solver.from_state(st, precision=gks.PREC_FP32_BULK)
    A.steps(0.01, 3)
    A.set_state(st.W, st.Wx, st.Wy)     # back to the initial state
    A.steps(0.01, 2)
    B = gks.Solver.from_state(st, precision=gks.PREC_FP32_BULK)
    B.steps(0.01, 2)
    for a, b in zip(A.get_state(), B.get_state()):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("make", [lambda: inputs.isentropic_vortex_2d(40, order=8, ny=36),
                                  lambda: inputs.shear_layer_2d(32),
                                  lambda: inputs.sod_1d(300, order=8, recon=1)],
                         ids=["vortex_linear", "shear_ns_wenoz", "sod_1d"])
def test_fp32_bulk_restart_continues_bit_for_bit(make):
    """The float mirror is a function of the FP64 state (the stage-2 update writes it exactly as
    set_state builds it), so a run stopped after two steps and restarted from its FP64 state in
    a new context continues bit for bit."""
    st = make()
    A = gks.Solver.from_state(st, precision=gks.PREC_FP32_BULK)
    dt = 0.3 / A.max_wavespeed()
    A.steps(dt, 4)
    B = gks.Solver.from_state(st, precision=gks.PREC_FP32_BULK)
    B.steps(dt, 2)
    C = gks.Solver.from_state(st, precision=gks.PREC_FP32_BULK)
    C.set_state(*B.get_state())
    C.steps(dt, 2)
    for a, c in zip(A.get_state(), C.get_state()):
        if a is not None:
            assert np.array_equal(a, c)


@pytest.mark.parametrize("prec", [gks.PREC_FP64, gks.PREC_FP32_BULK], ids=["fp64", "fp32"])
def test_viscous_shear_wave_decay_on_gpu(prec):
    # the decay exp(-nu k^2 t) of a transverse shear wave, 64 cells across: the scheme's
    # first-order-in-time viscous error is ~2.5e-4 here (7e-4 at 16 cells on the oracle)
    st = inputs.shear_wave_2d(16, 64)
    S = gks.Solver.from_state(st, precision=prec)
    t, T = 0.0, st.t_end
    while t < T - 1e-14:
        dt = min(0.3 / S.max_wavespeed(), T - t)
        S.step(dt)
        t += dt
    W = S.get_state()[0]
    ratio = inputs.shear_wave_amplitude(st, W) / inputs.shear_wave_amplitude(st, st.W)
    exact = math.exp(-st.mu * st.meta["k"] ** 2 * T)
    assert abs(ratio / exact - 1.0) < 4e-4, ratio / exact - 1.0

