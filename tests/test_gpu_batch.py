"""Batched form: many problems of uneven size in one persistent launch per step.

A problem advanced in a batch runs the same device code as the same problem advanced alone
by the FP32-bulk form.  The two are compiled into different kernels, and the compiler's
choice of fusing a multiply and an add into one FMA depends on the surrounding code, so the
two agree to single-precision rounding of the FP32 parts, not bitwise.  At a discontinuity
the single-precision flux delta is as large as the flux itself, so the differences reach
~2e-7 of W there (measured on a GB300); the bounds below (W within 1e-6 relative, slopes
within 1e-5 of max|W|/dx) stay under the FP32-bulk form's own bounds against FP64.  Within the batch the result does
not depend on the tile shape, the occupancy or the order in which tiles are handed out
(bitwise).  The autotuner must not change the state; a dependency wait that cannot be
satisfied must end in GKS_ETIMEOUT, not a hang.
"""
import numpy as np
import pytest

from paper_1901_00261_gb300 import gks, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gks.lib()


def mixed_states(n=10, seed=5, n1=(100, 3000), n2=(16, 96)):
    specs = inputs.batch_specs(n, seed=seed, n1_range=n1, n2_range=n2)
    return [inputs.build_problem(s) for s in specs]


TOL_W, TOL_SLOPE = 1e-6, 1e-5


def assert_close_to_alone(got, ref, st, what):
    W = ref[0]
    for k, (a, b) in enumerate(zip(got, ref)):
        if b is None:
            continue
        for v in range(b.shape[0]):
            scale = np.abs(b[v]).max()
            if k > 0:
                h = st.dx if k == 1 else st.dy
                scale = max(scale, np.abs(W[v]).max() / h)
            err = np.abs(a[v] - b[v]).max() / max(scale, 1e-300)
            assert err <= (TOL_W if k == 0 else TOL_SLOPE), f"{what}: array {k} var {v}: {err:.3e}"


def run_alone(st, dt, nsteps):
    S = gks.Solver.from_state(st, precision=gks.PREC_FP32_BULK)
    S.steps(dt, nsteps)
    return S.get_state()


def dts_of(states):
    out = []
    for st in states:
        S = gks.Solver.from_state(st, precision=gks.PREC_FP32_BULK)
        out.append(0.3 / S.max_wavespeed())
    return np.array(out)


def set_config_fitting(B, fpt, bps):
    """Tile shape `fpt` with the most resident blocks per SM up to `bps` that fit (taller tiles
    take more shared memory)."""
    for b in range(bps, 0, -1):
        try:
            B.set_config(fpt, b)
            return b
        except gks.GksError:
            continue
    raise AssertionError(f"no block count fits tile shape {fpt}")


@pytest.mark.parametrize("fpt", [1, 2, 4])
def test_batch_matches_individual_runs(fpt):
    states = mixed_states()
    dts = dts_of(states)
    B = gks.Batch(states)
    _, maxb = B.config()
    set_config_fitting(B, fpt, maxb)
    B.steps(dts, 3)
    for k, st in enumerate(states):
        assert_close_to_alone(B.get_state(k), run_alone(st, dts[k], 3), st,
                              f"problem {k} ({st.name}, {st.nx}x{st.ny})")


def test_batch_tile_shapes_and_occupancy_agree():
    states = mixed_states(6, seed=9)
    dts = dts_of(states)
    results = []
    for fpt, bps in ((1, 1), (2, 2), (1, 3), (4, 1), (4, 2)):
        B = gks.Batch(states)
        set_config_fitting(B, fpt, min(bps, B.config()[1]))
        B.steps(dts, 2)
        results.append([B.get_state(k) for k in range(len(states))])
    for other in results[1:]:
        for ga, gb in zip(results[0], other):
            for a, b in zip(ga, gb):
                if b is not None:
                    assert np.array_equal(a, b)


def test_batch_class_with_2d_weno_and_navier_stokes():
    states = [inputs.isentropic_vortex_2d(40, order=8, recon=1, ny=33),
              inputs.shear_layer_2d(32),
              inputs.sod_1d(257, order=6, recon=1),
              inputs.isentropic_vortex_2d(29, order=6, recon=0)]
    dts = dts_of(states)
    B = gks.Batch(states)
    B.steps(dts, 2)
    for k, st in enumerate(states):
        assert_close_to_alone(B.get_state(k), run_alone(st, dts[k], 2), st, f"problem {k}")


def test_autotune_restores_state_and_keeps_results():
    states = mixed_states(8, seed=11)
    dts = dts_of(states)
    B = gks.Batch(states)
    report = B.autotune(dts, steps=2)
    assert "chosen" in report
    fpt, bps = B.config()
    assert fpt in (1, 2, 4) and bps >= 1
    assert any(line.startswith("4 ") for line in report.splitlines())   # 32 x 16 tiles were timed
    B.steps(dts, 2)
    for k, st in enumerate(states):
        assert_close_to_alone(B.get_state(k), run_alone(st, dts[k], 2), st, f"problem {k}")


def test_batch_max_wavespeed_matches_single():
    states = mixed_states(5, seed=2)
    B = gks.Batch(states)
    ws = B.max_wavespeed()
    for k, st in enumerate(states):
        S = gks.Solver.from_state(st, precision=gks.PREC_FP32_BULK)
        assert ws[k] == S.max_wavespeed()


def test_batch_missing_producer_times_out_and_recovers():
    """A wait on a producer that never comes runs out of its (short) budget: the step ends,
    gks_batch_sync reports GKS_ETIMEOUT, and after a reset the batch steps normally."""
    states = mixed_states(4, seed=3, n1=(100, 300), n2=(16, 24))
    dts = dts_of(states)
    B = gks.Batch(states)
    B.debug_missing_producer(1, 0, 0.2)
    B.steps(dts, 1)
    with pytest.raises(gks.GksError) as ei:
        B.sync()
    assert ei.value.code == gks.GKS_ETIMEOUT
    B.reset()
    for k, st in enumerate(states):
        B.set_state(k, st.W, st.Wx, st.Wy)
    B.steps(dts, 1)
    B.sync()
    for k, st in enumerate(states):
        assert_close_to_alone(B.get_state(k), run_alone(st, dts[k], 1), st, f"problem {k}")


def test_batch_freezes_a_nonphysical_problem_and_keeps_the_rest():
    """Toro's test 3 data (p 1000 | 0.01; the oracle meets a negative energy after one step at
    8th order, WENO-Z, N = 200) among healthy problems: the failing problem is reported by
    index and frozen, every other problem advances exactly as if it were alone, and
    set_state puts the failed problem back in service."""
    bad = inputs.riemann_1d(200, (1.0, 0.0, 1000.0), (1.0, 0.0, 0.01), 0.0, 1.0, 0.5, 1.4, 8, 1)
    good = mixed_states(4, seed=7, n1=(100, 400), n2=(16, 32))
    states = good[:2] + [bad] + good[2:]
    dts = dts_of(states)
    B = gks.Batch(states)
    B.steps(dts, 3)
    with pytest.raises(gks.GksError) as ei:
        B.sync()
    assert ei.value.code == gks.GKS_ENONPHYSICAL and "2" in str(ei.value)
    status = B.problem_status()
    assert list(status) == [0, 0, gks.GKS_ENONPHYSICAL, 0, 0]
    for k, st in enumerate(states):
        if k != 2:
            assert_close_to_alone(B.get_state(k), run_alone(st, dts[k], 3), st, f"problem {k}")
    with pytest.raises(gks.GksError):
        B.get_state(2)
    calm = inputs.riemann_1d(200, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.0, 1.0, 0.5, 1.4, 8, 1)
    B.set_state(2, calm.W, calm.Wx)
    assert list(B.problem_status()) == [0] * 5
    dt2 = dts.copy()
    dt2[2] = dts_of([calm])[0]
    B.steps(dt2, 1)
    B.sync()
    assert_close_to_alone(B.get_state(2), run_alone(calm, dt2[2], 1), calm, "restarted problem")


# FP32-bulk bounds of tests/test_gpu_fp32.py per problem class: (W, slopes), per step from
# identical input against the FP64 reference (here the oracle), slopes relative to the scale
# max|W|/dx of their difference quotient.
ORACLE_BOUNDS = {"linear": (3e-8, 3e-7), "wenoz_1d": (2e-6, 2e-6), "wenoz_2d": (3e-7, 2e-6),
                 "ns": (2e-5, 2e-5)}


def _oracle_step(st, W, Wx, Wy, dt):
    import oracle
    O = oracle.Solver(st.nx, st.ny, st.gamma, st.mu, st.Pr, st.order, st.recon, st.bc_x, st.bc_y,
                      st.x0, st.x1, st.y0, st.y1)
    O.set_state(W, Wx, Wy)
    O.step(dt)
    return O.get_state()


def test_batch_members_match_the_oracle_per_step():
    """A mixed batch (1D WENO-Z Riemann problems from the batched workload's recipe, 2D
    linear vortices, both orders, plus a 2D WENO-Z vortex and a Navier-Stokes shear layer):
    for two consecutive steps each member's batch step from its current state is compared
    with the FP64 oracle's step from the same state, within the FP32-bulk form's bounds."""
    specs = inputs.batch_specs(8, seed=13, n1_range=(100, 400), n2_range=(16, 40))
    states = [inputs.build_problem(s) for s in specs]
    states += [inputs.isentropic_vortex_2d(24, order=8, recon=1, ny=20), inputs.shear_layer_2d(24)]
    kinds = []
    for st in states:
        if st.mu > 0:
            kinds.append("ns")
        elif st.recon == 1:
            kinds.append("wenoz_1d" if st.ny == 1 else "wenoz_2d")
        else:
            kinds.append("linear")
    assert {"linear", "wenoz_1d"} <= set(kinds) and {6, 8} <= {st.order for st in states}
    dts = dts_of(states)
    B = gks.Batch(states)
    for step in range(2):
        before = [B.get_state(k) for k in range(len(states))]
        B.steps(dts, 1)
        for k, st in enumerate(states):
            ref = _oracle_step(st, *before[k], dts[k])
            got = B.get_state(k)
            tw, ts = ORACLE_BOUNDS[kinds[k]]
            Wr = ref[0]
            for a_i, (a, b) in enumerate(zip(got, ref)):
                if b is None:
                    continue
                for v in range(b.shape[0]):
                    scale = np.abs(b[v]).max()
                    if a_i > 0:
                        scale = max(scale, np.abs(Wr[v]).max() / (st.dx if a_i == 1 else st.dy))
                    err = np.abs(a[v] - b[v]).max() / max(scale, 1e-300)
                    assert err <= (tw if a_i == 0 else ts), \
                        f"step {step} problem {k} ({kinds[k]}, {st.nx}x{st.ny}) array {a_i} var {v}: {err:.3e}"


def test_batch_with_reflecting_walls():
    """Walled problems (1D wall impact; 2D box pulses between walls on one or both axes,
    linear and WENO-Z) in one batch with a periodic vortex: the batch then runs the persistent
    kernel compiled with the wall signs.  Every member matches its standalone FP32-bulk run,
    and a walled member's step matches the oracle's within the FP32-bulk bounds."""
    states = [inputs.wall_impact_1d(300, order=8),
              inputs.box_pulse_2d(40, ny=36),
              inputs.box_pulse_2d(32, ny=28, order=6, recon=1),
              inputs.box_pulse_2d(30, ny=35, recon=1, bc_x=1),
              inputs.box_pulse_2d(33, ny=27, order=6, bc_y=0),
              inputs.isentropic_vortex_2d(24, order=8, recon=0, ny=20)]
    dts = dts_of(states)
    for fpt in (1, 2, 4):
        B = gks.Batch(states)
        set_config_fitting(B, fpt, B.config()[1])
        B.steps(dts, 3)
        for k, st in enumerate(states):
            assert_close_to_alone(B.get_state(k), run_alone(st, dts[k], 3), st,
                                  f"fpt {fpt} problem {k} ({st.name}, {st.nx}x{st.ny})")
    st = states[1]
    B = gks.Batch(states)
    before = B.get_state(1)
    B.steps(dts, 1)
    ref = _oracle_step(st, *before, dts[1])
    got = B.get_state(1)
    tw, ts = ORACLE_BOUNDS["linear"]
    for a_i, (a, b) in enumerate(zip(got, ref)):
        for v in range(b.shape[0]):
            scale = np.abs(b[v]).max()
            if a_i > 0:
                scale = max(scale, np.abs(ref[0][v]).max() / (st.dx if a_i == 1 else st.dy))
            err = np.abs(a[v] - b[v]).max() / max(scale, 1e-300)
            assert err <= (tw if a_i == 0 else ts), f"array {a_i} var {v}: {err:.3e}"


def test_batch_rejects_isothermal_walls():
    st = inputs.box_pulse_2d(16, ny=16)
    st.bc_x = 3
    with pytest.raises(gks.GksError):
        gks.Batch([st])
