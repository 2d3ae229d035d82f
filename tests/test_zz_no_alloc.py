"""gks_step_1d_static: the step for callers that cannot allocate device memory.

Such callers (code inside a memory pool it does not own, a host application that forbids
device allocation after start-up, a real-time loop) pass device buffers for the state
and the result; the library keeps its scratch in a static device array.  This checks,
through the C ABI, that two calls in a row (the second one in place) give the same state as
the allocating entry point (gks_create / gks_step), Euler and Navier-Stokes, within the
parity tolerance of the other GPU tests, that the device's free memory does not move across
a call, and that a grid larger than the static scratch and non-finite parameters are refused.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1901_00261_gb300 import gks, inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_header_limit_matches_binding():
    text = open(os.path.join(ROOT, "include", "gks.h")).read()
    m = re.search(r"#define\s+GKS_STATIC_MAX_NX\s+(\d+)", text)
    assert m and int(m.group(1)) == gks.STATIC_MAX_NX


def _state(order, recon, N, case):
    if case == "wall":
        return inputs.wall_impact_1d(N, order=order, recon=recon)
    if case.endswith("wave"):
        st = inputs.density_wave_1d(N, order=order, recon=recon)
    else:
        st = inputs.sod_1d(N, order=order, recon=recon)
    # Navier-Stokes: the viscous kernel instances and the Prandtl fix (viscosities at which
    # the scheme stays physical on these data; the oracle fails alike beyond them)
    if case == "viscous_sod":
        st.mu, st.Pr = 2e-4, 0.72
    elif case == "viscous_wave":
        st.mu, st.Pr = 1e-3, 0.72
    return st


@pytest.mark.parametrize("order,recon,N,case", [(6, 0, 80, "wave"), (8, 1, 1000, "sod"),
                                                (8, 1, 400, "wall"), (6, 1, 300, "viscous_sod"),
                                                (8, 0, 200, "viscous_wave")])
def test_static_step_matches_allocating_entry_point(order, recon, N, case):
    """Two calls in a row, the second one in place (outputs aliasing the inputs), against
    gks_create / gks_step with the same physics; the device's free memory does not change
    across the second call (no allocation by the library or anything it calls)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = gks.lib()
    st = _state(order, recon, N, case)
    ref = gks.Solver.from_state(st)
    dt = 0.3 / ref.max_wavespeed()

    W = torch.from_numpy(st.W.reshape(3, N).copy()).cuda()
    Wx = torch.from_numpy(st.Wx.reshape(3, N).copy()).cuda()
    Wo = torch.empty_like(W)
    Wxo = torch.empty_like(W)
    stream = torch.cuda.current_stream().cuda_stream
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731

    def call(a, ax, b, bx):
        rc = L.gks_step_1d_static(p(a), p(ax), p(b), p(bx), N, st.gamma, st.mu, st.Pr, st.x0,
                                  st.x1, st.bc_x, order, recon, dt, ctypes.c_void_p(stream))
        assert rc == gks.GKS_OK, L.gks_static_last_error().decode()

    def check(a_t, ax_t, tag):
        ref.step(dt)
        Wr, Wxr, _ = ref.get_state()
        a, ax = a_t.cpu().numpy().reshape(3, 1, N), ax_t.cpu().numpy().reshape(3, 1, N)
        for v in range(3):
            sw = np.abs(Wr[v]).max()
            assert np.abs(a[v] - Wr[v]).max() <= TOL * sw, f"{tag} W[{v}]"
            sx = max(np.abs(Wxr[v]).max(), sw / st.dx)
            assert np.abs(ax[v] - Wxr[v]).max() <= TOL * sx, f"{tag} Wx[{v}]"

    call(W, Wx, Wo, Wxo)                       # first call: separate outputs
    check(Wo, Wxo, "call 1")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    call(Wo, Wxo, Wo, Wxo)                     # second call: in place
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    check(Wo, Wxo, "call 2 (in place)")
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"


def test_static_step_rejects_oversize_grid():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = gks.lib()
    N = gks.STATIC_MAX_NX + 1
    W = torch.ones((3, N), dtype=torch.float64, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    rc = L.gks_step_1d_static(p(W), p(W), p(W), p(W), N, 1.4, 0.0, 1.0, 0.0, 1.0, 0, 6, 0, 1e-3, None)
    assert rc == gks.GKS_EINVAL
    assert "GKS_STATIC_MAX_NX" in L.gks_static_last_error().decode()


def test_static_step_rejects_non_finite_parameters():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = gks.lib()
    W = torch.ones((3, 16), dtype=torch.float64, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    inf, nan = float("inf"), float("nan")
    for gamma, mu, Pr, x0, x1 in [(inf, 0.0, 1.0, 0.0, 1.0), (1.4, inf, 1.0, 0.0, 1.0),
                                  (1.4, 0.0, inf, 0.0, 1.0), (1.4, 0.0, 1.0, -inf, 1.0),
                                  (1.4, 0.0, 1.0, 0.0, inf), (nan, 0.0, 1.0, 0.0, 1.0)]:
        rc = L.gks_step_1d_static(p(W), p(W), p(W), p(W), 16, gamma, mu, Pr, x0, x1, 0, 6, 0,
                                  1e-3, None)
        assert rc == gks.GKS_EINVAL, (gamma, mu, Pr, x0, x1)
