"""gks_step_1d_static: the step for callers that cannot allocate device memory.

Such callers (code inside a memory pool it does not own, a host application that forbids
device allocation after start-up, a real-time loop) pass device buffers for the state
and the result; the library keeps its scratch in a static device array.  This checks,
through the C ABI, that two calls in a row give the same state as the allocating entry
point (gks_create / gks_step), within the parity tolerance of the other GPU tests, and
that a grid larger than the static scratch is refused.
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


@pytest.mark.parametrize("order,recon,N,wall", [(6, 0, 80, False), (8, 1, 1000, False),
                                                (8, 1, 400, True)])
def test_static_step_matches_allocating_entry_point(order, recon, N, wall):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = gks.lib()
    if wall:
        st = inputs.wall_impact_1d(N, order=order, recon=recon)
    elif recon == 0:
        st = inputs.density_wave_1d(N, order=order, recon=recon)
    else:
        st = inputs.sod_1d(N, order=order, recon=recon)
    ref = gks.Solver.from_state(st)
    dt = 0.3 / ref.max_wavespeed()

    W = torch.from_numpy(st.W.reshape(3, N).copy()).cuda()
    Wx = torch.from_numpy(st.Wx.reshape(3, N).copy()).cuda()
    Wo = torch.empty_like(W)
    Wxo = torch.empty_like(W)
    stream = torch.cuda.current_stream().cuda_stream
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    for call in range(2):
        rc = L.gks_step_1d_static(p(W), p(Wx), p(Wo), p(Wxo), N, st.gamma, 0.0, 1.0, st.x0, st.x1,
                                  st.bc_x, order, recon, dt, ctypes.c_void_p(stream))
        assert rc == gks.GKS_OK, L.gks_static_last_error().decode()
        ref.step(dt)
        Wr, Wxr, _ = ref.get_state()
        a, ax = Wo.cpu().numpy().reshape(3, 1, N), Wxo.cpu().numpy().reshape(3, 1, N)
        for v in range(3):
            sw = np.abs(Wr[v]).max()
            assert np.abs(a[v] - Wr[v]).max() <= TOL * sw, f"call {call} W[{v}]"
            sx = max(np.abs(Wxr[v]).max(), sw / st.dx)
            assert np.abs(ax[v] - Wxr[v]).max() <= TOL * sx, f"call {call} Wx[{v}]"
        W, Wo = Wo, W
        Wx, Wxo = Wxo, Wx


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
