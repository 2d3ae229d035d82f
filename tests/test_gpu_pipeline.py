"""The pipelined host-to-host step (gks_step_host_async) against the synchronous calls.

Several calls are in flight at once (three device slots, two copy streams); each result must
equal, bit for bit, set_state + step + get_state of the same input on a second solver (the
same kernels on the same numbers), for both forms, 1D and 2D, with dt changing between
calls.  The context's own state must be left alone, and a later ordinary step must still see
its own float mirror (the pipelined steps borrow it).
"""
import numpy as np
import pytest

from paper_1901_00261_gb300 import gks, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    gks.lib()
    return t


def pinned(torch, shape):
    return torch.empty(shape, dtype=torch.float64).pin_memory().numpy()


def perturbed(st, k):
    """Input k: the state with its density and energy scaled by 1 + 1e-3 k (still physical)."""
    s = np.ones((st.W.shape[0],) + (1,) * (st.W.ndim - 1))
    s[0] = s[-1] = 1.0 + 1e-3 * k
    return [st.W * s, st.Wx * s] + ([st.Wy * s] if st.Wy is not None else [])


CASES = [
    ("2D linear vortex 64x48 fp32", lambda: inputs.isentropic_vortex_2d(64, ny=48), gks.PREC_FP32_BULK),
    ("2D linear vortex 64x48 fp64", lambda: inputs.isentropic_vortex_2d(64, ny=48), gks.PREC_FP64),
    ("2D WENO-Z vortex 40x40 fp32", lambda: inputs.isentropic_vortex_2d(40, recon=1), gks.PREC_FP32_BULK),
    ("1D WENO-Z Sod 300 fp32", lambda: inputs.sod_1d(300), gks.PREC_FP32_BULK),
    ("1D WENO-Z Sod 300 fp64", lambda: inputs.sod_1d(300), gks.PREC_FP64),
]


@pytest.mark.parametrize("name,make,prec", CASES, ids=[c[0] for c in CASES])
def test_pipelined_steps_equal_synchronous_steps(torch, name, make, prec):
    st = make()
    G = gks.Solver.from_state(st, precision=prec)
    own = G.get_state()
    R = gks.Solver.from_state(st, precision=prec)
    dt0 = 0.3 / G.max_wavespeed()
    n = 7
    ins, outs, dts = [], [], []
    for k in range(n):
        arrs = perturbed(st, k)
        ins.append([pinned(torch, G.shape) for _ in arrs])
        for dst, src in zip(ins[-1], arrs):
            dst[...] = src.reshape(G.shape)
        outs.append([pinned(torch, G.shape) for _ in arrs])
        dts.append(dt0 * (1.0 if k % 2 == 0 else 0.5))
    for k in range(n):
        G.step_host_async(ins[k], outs[k], dts[k])
    G.sync()
    for k in range(n):
        R.set_state(*ins[k])
        R.step(dts[k])
        ref = R.get_state()
        for a, b in zip(outs[k], ref):
            assert np.array_equal(a, b), f"{name}: call {k}"
    # the context's own state is untouched, and an ordinary step from it matches a fresh
    # solver's (the float mirror of the own state is rebuilt after the pipelined steps)
    for a, b in zip(G.get_state(), own):
        if b is not None:
            assert np.array_equal(a, b)
    G.step(dt0)
    F = gks.Solver.from_state(st, precision=prec)
    F.step(dt0)
    for a, b in zip(G.get_state(), F.get_state()):
        if b is not None:
            assert np.array_equal(a, b), f"{name}: own step after the pipeline"


def test_pipelined_rejects_bad_arrays(torch):
    st = inputs.isentropic_vortex_2d(16)
    G = gks.Solver.from_state(st, precision=gks.PREC_FP32_BULK)
    good = [np.zeros(G.shape) for _ in range(3)]
    with pytest.raises(ValueError):
        G.step_host_async([np.zeros((4, 16, 15))] + good[1:], good, 0.01)
    with pytest.raises(gks.GksError):
        G.step_host_async(good, [np.zeros(G.shape) for _ in range(3)], -1.0)
