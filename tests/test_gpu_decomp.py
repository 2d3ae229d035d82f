"""Device-resident row-split decomposition (decomp.DeviceDecomposedRun) on one GPU: two slabs,
each a gks.Solver holding its rows plus 4 halo rows on the device, advanced in one process
with the halo exchange done in-process (each slab's packed boundary blocks handed to the
other): the assembled result equals the single-domain GPU run bit for bit, in the FP64 and
the FP32-bulk forms (the FP32-bulk float mirror is a function of the FP64 state, so halo rows
refreshed from FP64 rows carry the same mirror as the single-domain run).  (The all_gather itself is exercised by the gloo ranks of tests/test_decomp.py; two ranks on
one GPU are not run.)  Also the row copies themselves: gks_set_rows_device /
gks_get_rows_device against set_state / get_state."""
import numpy as np
import pytest

from paper_1901_00261_gb300 import decomp, gks, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gks.lib()


def _case(name):
    if name == "vortex_linear":
        return inputs.isentropic_vortex_2d(40, order=8, recon=0, ny=36)
    if name == "vortex_weno":
        return inputs.isentropic_vortex_2d(32, order=6, recon=1, ny=28)
    if name == "shear_ns":
        return inputs.shear_layer_2d(32)
    return inputs.box_pulse_2d(26, ny=30)   # walls in x and y


def _factory(st, prec):
    def make(ny_ext, y0, y1, bc_y):
        return gks.Solver(st.nx, ny_ext, st.gamma, st.mu, st.Pr, st.order, st.recon, st.x0, st.x1,
                          y0, y1, st.bc_x, bc_y, precision=prec)
    return make


@pytest.mark.parametrize("prec", [gks.PREC_FP64, gks.PREC_FP32_BULK])
@pytest.mark.parametrize("name", ["vortex_linear", "vortex_weno", "shear_ns", "box_walls"])
def test_device_slabs_equal_the_single_domain_run(name, prec):
    st = _case(name)
    nr = 2
    runs = [decomp.DeviceDecomposedRun(st.W, st.Wx, st.Wy, st.y0, st.y1, st.bc_y,
                                       _factory(st, prec), r, nr) for r in range(nr)]
    S = gks.Solver.from_state(st, precision=prec)
    dt = 0.3 / S.max_wavespeed()
    for _ in range(4):
        S.step(dt)
        for r in runs:
            r.solver.step(dt)
        parts = [r.pack().clone() for r in runs]
        for r in runs:
            r.unpack(parts)
    own = [r.own_state() for r in runs]
    got = [np.concatenate([o[k] for o in own], axis=1) for k in range(3)]
    ref = S.get_state()
    for k in range(3):
        assert np.array_equal(got[k], ref[k]), f"array {k}: max diff {np.abs(got[k] - ref[k]).max():.3e}"


@pytest.mark.parametrize("prec", [gks.PREC_FP64, gks.PREC_FP32_BULK])
def test_row_copies(prec):
    import torch
    st = inputs.isentropic_vortex_2d(24, order=8, recon=0, ny=20)
    S = gks.Solver.from_state(st, precision=prec)
    buf = torch.empty((3, 4, 5, st.nx), dtype=torch.float64, device="cuda")
    S.get_rows_device(7, 5, buf.data_ptr())
    S.sync()
    b = buf.cpu().numpy()
    for k, A in enumerate((st.W, st.Wx, st.Wy)):
        assert np.array_equal(b[k], A[:, 7:12, :])
    # rows written back from another state: the step afterwards is that of the combined state
    other = inputs.isentropic_vortex_2d(24, t=0.3, order=8, recon=0, ny=20)
    src = torch.from_numpy(np.stack([A[:, 3:9, :] for A in (other.W, other.Wx, other.Wy)])).cuda()
    S.set_rows_device(3, 6, src.data_ptr())
    comb = [A.copy() for A in (st.W, st.Wx, st.Wy)]
    for k, A in enumerate((other.W, other.Wx, other.Wy)):
        comb[k][:, 3:9, :] = A[:, 3:9, :]
    R = gks.Solver(st.nx, st.ny, st.gamma, st.mu, st.Pr, st.order, st.recon, st.x0, st.x1, st.y0,
                   st.y1, st.bc_x, st.bc_y, precision=prec)
    R.set_state(*comb)
    dt = 0.3 / R.max_wavespeed()
    S.step(dt)
    R.step(dt)
    for a, b in zip(S.get_state(), R.get_state()):
        assert np.array_equal(a, b)
    with pytest.raises(gks.GksError):
        S.get_rows_device(18, 3, buf.data_ptr())   # beyond the last row
