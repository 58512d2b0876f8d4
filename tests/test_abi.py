"""The C ABI library loads and exports every entry point of include/gg.h, and
host-side argument validation rejects bad input before any device work.
No GPU is needed: only calls that fail validation are made."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2006_01748_gb300 import build, gg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return gg.lib()


def header_functions():
    src = open(os.path.join(ROOT, "include", "gg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gg_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ["gg_create", "gg_step", "gg_adjoint", "gg_read", "gg_write", "gg_diagnostics",
                     "gg_destroy", "gg_batch_create", "gg_batch_step", "gg_batch_read", "gg_batch_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in header_functions() if getattr(lib, n, None) is None]
    assert not missing, f"declared in include/gg.h but not exported: {missing}"


def test_binding_covers_the_header():
    assert set(header_functions()) <= set(gg.exported_symbols())


def test_error_strings(lib):
    assert gg.gg_error_string(0) == "ok"
    for code in range(-8, 0):
        assert gg.gg_error_string(code) != "unknown status"


def _create(grid, params, n=4):
    a = np.ones(n)
    ptr = a.ctypes.data_as(ctypes.c_void_p)
    return gg.gg_create(grid, params, ptr, ptr, ptr, ptr, ptr, ptr)


@pytest.mark.parametrize("bad", [
    dict(nx=0), dict(ny=-3), dict(delta=-1.0), dict(D=float("nan")), dict(cfl=1.5),
    dict(precision=7), dict(flags=64), dict(steps_per_pass=9), dict(adapt_every=-1), dict(dt=-1.0),
    dict(adapt_every=5, dt=1e-6),
])
def test_host_validation_rejects_bad_arguments(lib, bad):
    grid = gg.gg_grid(bad.get("nx", 2), bad.get("ny", 2), 1.0, 1.0)
    p = gg.make_params(bad.get("delta", 1.0), 1.0, bad.get("D", 1e-3), 70.0, cfl=bad.get("cfl", 0.9),
                       dt=bad.get("dt", 0.0))
    if "precision" in bad:
        p.precision = bad["precision"]
    if "flags" in bad:
        p.flags = bad["flags"]
    if "steps_per_pass" in bad:
        p.steps_per_pass = bad["steps_per_pass"]
    if "adapt_every" in bad:
        p.adapt_every = bad["adapt_every"]
    rc, sim = _create(grid, p)
    assert rc == gg.GG_ERR_ARG
    assert not sim.value
    assert gg.gg_last_error(None)


def test_null_field_pointer_rejected(lib):
    grid = gg.gg_grid(2, 2, 1.0, 1.0)
    p = gg.make_params(1.0, 1.0, 1e-3, 70.0)
    out = ctypes.c_void_p()
    rc = lib.gg_create(ctypes.byref(grid), ctypes.byref(p), None, None, None, None, None, None, None,
                       ctypes.byref(out))
    assert rc == gg.GG_ERR_ARG


def test_null_handles_are_rejected(lib):
    assert lib.gg_step(None, 1) == gg.GG_ERR_ARG
    assert lib.gg_read(None, 0, None, 0, 1) == gg.GG_ERR_ARG
    assert lib.gg_front_rays(None, 0, 0, 0.5, 0.5, 0.01, None) == gg.GG_ERR_ARG
    assert lib.gg_front_speed(None, 0, 0, 1, 0.5, 0.5, 0.01, None, None, None) == gg.GG_ERR_ARG
    assert lib.gg_adjoint_release(None) == gg.GG_ERR_ARG
    assert lib.gg_batch_set_plan(None, 0, 1, 0) == gg.GG_ERR_ARG
    assert lib.gg_destroy(None) == gg.GG_OK
    assert lib.gg_dt(None) == 0.0
    assert lib.gg_time(None) == 0.0
