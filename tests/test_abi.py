"""The C-ABI library builds, loads and exports every symbol include/gks.h declares; host-side
argument checks run without a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_1901_00261_gb300 import gks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    syms = set()
    for name in os.listdir(os.path.join(ROOT, "include")):
        if not name.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", name)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(gks_[a-z0-9_]+)\s*\(", text):
            syms.add(m.group(1))
    return syms


def test_library_exports_every_declared_symbol():
    L = gks.lib()
    syms = declared_symbols()
    assert "gks_create" in syms and "gks_step" in syms
    missing = [s for s in sorted(syms) if not hasattr(L, s)]
    assert not missing, missing
    # and the binding knows every one of them
    assert set(gks.SIGNATURES) >= syms


def test_default_opts():
    o = gks.default_opts()
    assert (o.x0, o.x1, o.bc_x, o.weno_eps, o.eps_tau, o.C_tau, o.use_graph) == (0.0, 1.0, 0, 1e-6, 0.01, 1.0, 1)
    assert o.tau_mode == 0 and o.stream is None and o.tan_mode == 0
    # the last fields: a layout mismatch between the header and the binding shows here
    assert list(o.wall_T) == [1.0] * 4 and list(o.wall_u) == [0.0] * 4 and o.coef_mode == 0


@pytest.mark.parametrize("change,msg", [
    (dict(bc_x=4), "bc must be"),
    (dict(bc_x=3, precision=1), "FP64 form only"),
    (dict(bc_y=3, wall_T=(1.0, 1.0, 0.0, 1.0)), "wall_T"),
    (dict(bc_x=3, wall_u=(0.0, float("nan"), 0.0, 0.0)), "wall_u"),
    (dict(bc_x=2, bc_y=3, wall_u=(0.0, 0.0, 0.0, 0.1)), "reflecting"),
    (dict(coef_mode=2), "coef_mode"),
    (dict(coef_mode=1, precision=1), "coef_mode 1"),
    (dict(coef_mode=1, tau_mode=1), "coef_mode 1"),
])
def test_create_rejects_invalid_walls(change, msg):
    L = gks.lib()
    o = gks.default_opts()
    for k, v in change.items():
        if k in ("wall_T", "wall_u"):
            for i, x in enumerate(v):
                getattr(o, k)[i] = x
        else:
            setattr(o, k, v)
    assert not L.gks_create(10, 10, 1.4, 0.01, 0.72, 6, 0, ctypes.byref(o))
    assert msg in gks.last_error()


def test_create_rejects_invalid_tau_mode():
    L = gks.lib()
    o = gks.default_opts()
    o.tau_mode = 2
    assert not L.gks_create(10, 1, 1.4, 0.0, 1.0, 6, 0, ctypes.byref(o))
    assert "tau_mode" in gks.last_error()


@pytest.mark.parametrize("args,msg", [
    ((4, 1, 1.4, 0.0, 1.0, 6, 0), "nx >= 5"),
    ((10, 3, 1.4, 0.0, 1.0, 6, 0), "ny == 1 or ny >= 5"),
    ((10, 1, 1.4, 0.0, 1.0, 7, 0), "order"),
    ((10, 1, 1.0, 0.0, 1.0, 6, 0), "gamma"),
    ((10, 1, 1.4, -1.0, 1.0, 6, 0), "mu"),
    ((10, 1, 1.4, 0.0, 0.0, 6, 0), "Pr"),
    ((10, 1, 1.4, 0.0, 1.0, 6, 2), "recon"),
])
def test_create_rejects_invalid_arguments(args, msg):
    L = gks.lib()
    h = L.gks_create(*args, None)
    assert not h
    assert msg in gks.last_error()


def test_null_context_calls_fail_cleanly():
    L = gks.lib()
    assert L.gks_step(None, 0.1) == gks.GKS_EINVAL
    assert L.gks_sync(None) == gks.GKS_EINVAL
    assert L.gks_step_host_async(None, None, None, None, None, None, None, 0.1) == gks.GKS_EINVAL
    assert L.gks_probe_time_coefs(None, 1, 0.1, None) == gks.GKS_EINVAL
    assert L.gks_probe_time_coefs_single(None, 1, 0.1, None) == gks.GKS_EINVAL
    assert L.gks_get_rows_device(None, 0, 1, None) == gks.GKS_EINVAL
    assert L.gks_probe_d2f(None, 1, None) == gks.GKS_EINVAL
    assert L.gks_set_rows_device(None, 0, 1, None) == gks.GKS_EINVAL
    assert L.gks_get_state(None, None, None, None) == gks.GKS_EINVAL
    L.gks_destroy(None)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(gks, "_lib", None)
    monkeypatch.setattr(gks._build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        gks.lib(build_if_missing=False)


@pytest.mark.parametrize("mutate,msg", [
    (dict(nx=4), "nx >= 5"),
    (dict(ny=3), "ny == 1 or ny >= 5"),
    (dict(order=7), "order"),
    (dict(recon=2), "recon"),
    (dict(gamma=1.0), "physics or domain"),
    (dict(x1=0.0), "physics or domain"),
    (dict(bc_x=3), "bc"),
])
def test_batch_create_rejects_invalid_problems(mutate, msg):
    """Problem validation happens before any device work, so it is checked here without a GPU;
    the offending problem is named by index."""
    L = gks.lib()
    good = dict(nx=64, ny=1, order=8, recon=1, gamma=1.4, mu=0.0, Pr=1.0,
                x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc_x=1, bc_y=1)
    bad = dict(good, **mutate)
    arr = (gks.Problem * 2)()
    for k, d in enumerate((good, bad)):
        arr[k] = gks.Problem(d["nx"], d["ny"], d["order"], d["recon"], d["gamma"], d["mu"], d["Pr"],
                             d["x0"], d["x1"], d["y0"], d["y1"], d["bc_x"], d["bc_y"])
    assert not L.gks_batch_create(2, arr, None)
    err = L.gks_batch_last_error().decode()
    assert "problem 1" in err and msg in err


def test_batch_create_rejects_empty_list():
    L = gks.lib()
    assert not L.gks_batch_create(0, None, None)
    assert "n >= 1" in L.gks_batch_last_error().decode()
