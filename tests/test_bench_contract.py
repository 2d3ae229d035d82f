"""Host-side pieces of bench.py's JSON contract, checked without a GPU: the roofline block of
every modelled launch (fields, arithmetic, the issue-rate entry beside it) and the window
problem that the oracle and both GPU forms share."""
import math

import numpy as np
import pytest

import bench
from paper_1901_00261_gb300 import inputs


@pytest.mark.parametrize("key", sorted(bench.KERNEL_MODEL))
def test_roofline_block_for_every_modelled_launch(key):
    path, form, name = key
    n, ms = 2048, 0.4
    issue_peak = 4 * 152 * 2070e6
    r = bench.roofline(form, name, ms, n, n, 8, 1.25e12, 73e12, issue_peak, path=path)
    assert r["bound"] in ("alu", "hbm") and r["kernel"] == name
    assert r["unit"] in ("TFLOP/s", "GB/s")
    assert math.isclose(r["frac"], r["achieved"] / r["peak"], rel_tol=1e-12)
    m = bench.KERNEL_MODEL[key]
    units = ((n + 1) * n) if m["unit"] == "face" else n * n
    if r["unit"] == "TFLOP/s":
        per_unit = m["f32"] if r.get("pipe") == "fp32" else m["f64"]
        assert math.isclose(r["achieved"], per_unit * units / (ms * 1e-3) / 1e12, rel_tol=1e-12)
    # the largest fraction is the headline; the rest, and the issue rate, sit beside it
    for o in r["other_bounds"]:
        if o["bound"] != "issue":
            assert o["frac"] <= r["frac"]
    issue = [o for o in r["other_bounds"] if o["bound"] == "issue"]
    assert len(issue) == ("winstr" in m)
    if issue:
        assert math.isclose(issue[0]["frac"], m["winstr"] / 32 * units / (ms * 1e-3) / issue_peak,
                            rel_tol=1e-12)
    assert (r["traffic"] is None) == ("traffic" not in m)


def test_roofline_without_model_reports_nothing_measured():
    r = bench.roofline("fp32", "x_faces_stage1", 0.4, 256, 256, 6, 1.25e12, 73e12)
    assert r["frac"] is None and r["achieved"] is None


def test_oracle_window_is_the_centre_of_the_workload():
    st = inputs.isentropic_vortex_2d(64)
    w = bench.window_state(st, 16)
    assert (w.nx, w.ny, w.bc_x, w.bc_y) == (16, 16, 1, 1)
    assert math.isclose(w.x1 - w.x0, 16 * st.dx) and math.isclose(w.y1 - w.y0, 16 * st.dy)
    assert np.array_equal(w.W, st.W[:, 24:40, 24:40])
    assert np.array_equal(w.Wy, st.Wy[:, 24:40, 24:40])


def test_single_thread_oracle_sample_restores_the_thread_count():
    import oracle
    before = oracle.get_threads()
    st = inputs.isentropic_vortex_2d(32)
    r = bench.cpu_single_thread(st, 0.01, budget_s=0.05, window=16)
    assert r["cores"] == 1 and r["value"] > 0 and r["kind"] == "oracle"
    assert oracle.get_threads() == before
