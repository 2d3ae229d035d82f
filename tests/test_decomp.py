"""Row-split domain decomposition of one problem (paper_1901_00261_gb300.decomp): the slab
geometry, and two gloo ranks on the CPU each advancing its slab (extended by the 4 halo
rows one two-stage step reaches) with the reference solver, exchanging halos once per step:
the assembled result equals the single-domain run bit for bit."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
from paper_1901_00261_gb300 import decomp  # noqa: E402


def test_split_rows_and_slab_geometry():
    assert decomp.split_rows(10, 3) == [(0, 4), (4, 7), (7, 10)]
    s = decomp.Slab(24, 0, 2, periodic_y=True)
    assert (s.j0, s.j1, s.lower, s.upper, s.hl, s.hu) == (0, 12, 1, 1, 4, 4)
    assert list(s.rows) == [20, 21, 22, 23] + list(range(16)) and s.own == slice(4, 16)
    assert s.local_bc_y(0) == 1
    t = decomp.Slab(24, 1, 2, periodic_y=False)
    assert (t.lower, t.upper, t.hl, t.hu) == (0, None, 4, 0)
    assert list(t.rows) == list(range(8, 24)) and t.local_bc_y(1) == 1 and t.local_bc_y(2) == 2
    with pytest.raises(ValueError):
        decomp.Slab(6, 0, 2, periodic_y=True)      # slabs thinner than the halo


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(name):
    from paper_1901_00261_gb300 import inputs
    if name == "vortex_weno_periodic":
        st = inputs.isentropic_vortex_2d(20, order=8, recon=1, ny=24)
    elif name == "shear_ns_periodic":
        st = inputs.shear_layer_2d(24)
    else:   # walls in y, transmissive x: the box pulse
        st = inputs.box_pulse_2d(18, ny=22)
    return st


def _dt(st):
    return 0.2 * min(st.dx, st.dy) / 3.0


def _oracle_factory(st):
    import oracle

    def make(ny_ext, y0, y1, bc_y):
        S = oracle.Solver(st.nx, ny_ext, st.gamma, st.mu, st.Pr, st.order, st.recon, st.bc_x, bc_y,
                          st.x0, st.x1, y0, y1)
        return S
    return make


def _rank(rank, world, port, name, steps, out):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, HERE)
    import oracle
    oracle.set_threads(1)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        st = _case(name)
        run = decomp.DecomposedRun(st.W, st.Wx, st.Wy, st.y0, st.y1, st.bc_y, _oracle_factory(st),
                                   rank, world, dist)
        dt = _dt(st)
        for _ in range(steps):
            run.step(dt)
        W, Wx, Wy = run.gather()
        if rank == 0:
            out["state"] = (W, Wx, Wy, dt)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["vortex_weno_periodic", "shear_ns_periodic", "box_walls"])
def test_two_slabs_equal_the_single_domain_run(name):
    steps = 3
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, _free_port(), name, steps, out), nprocs=world,
                           join=True, start_method="spawn")
        W, Wx, Wy, dt = out["state"]
    import oracle
    st = _case(name)
    O = oracle.Solver(st.nx, st.ny, st.gamma, st.mu, st.Pr, st.order, st.recon, st.bc_x, st.bc_y,
                      st.x0, st.x1, st.y0, st.y1)
    O.set_state(st.W, st.Wx, st.Wy)
    for _ in range(steps):
        O.step(dt)
    a, ax, ay = O.get_state()
    assert np.array_equal(W, a) and np.array_equal(Wx, ax) and np.array_equal(Wy, ay)
