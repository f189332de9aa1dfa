"""The C-ABI library builds for sm_103a, loads, exports every entry point
include/fsei.h declares, and rejects bad arguments at call time (host-side
validation only: no device computation is launched here)."""

import ctypes
import os
import re

import pytest

from paper_2103_15187_gb300 import build as fbuild
from paper_2103_15187_gb300 import fsei

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\S.*?\b(fsei_\w+)\s*\(", text, re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    fbuild.build()
    return fsei.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"fsei_grid_create", "fsei_step", "fsei_poisson_solve"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(fsei.EXPORTS) <= names


def test_version_and_error_string(lib):
    assert "sm_103a" in fsei.version()
    assert isinstance(lib.fsei_last_error(), bytes)


@pytest.mark.parametrize("shape,msg", [((10, 8, 8), "nx"), ((16, 10, 8), "ny"),
                                       ((16, 8, 4), "nz"), ((16, 8, 4096), "nz"),
                                       ((2, 8, 8), "nx")])
def test_bad_extents_rejected(lib, shape, msg):
    with pytest.raises(fsei.FseiError) as ei:
        fsei.Grid(*shape, 1.0, 1.0)
    assert ei.value.status == 2 and msg in str(ei.value)


def test_bad_arguments_rejected(lib):
    h = ctypes.c_void_p()
    assert lib.fsei_grid_create(None, ctypes.byref(h)) == 1
    with pytest.raises(fsei.FseiError) as ei:
        fsei.Grid(16, 8, 8, -1.0, 1.0)
    assert ei.value.status == 1
    with pytest.raises(fsei.FseiError):
        fsei.Grid(16, 8, 8, 1.0, 1.0, zbc=1, zfaces=[0, 1, 1, 2, 3, 4, 5, 6, 7])
    # NULL handle / state to the step and the Poisson solve
    prm = fsei.StepParams(100.0, 1e-3, 0.0, 1.5, -0.5, (ctypes.c_double * 3)())
    assert lib.fsei_step(None, None, None, None, None, ctypes.byref(prm), 1, None, None) == 1
    assert lib.fsei_poisson_solve(None, None, None, None) == 1
    lib.fsei_grid_destroy(None)


def test_missing_library_fails_loudly(tmp_path):
    saved = fsei._lib
    try:
        fsei._lib = None
        with pytest.raises(fsei.FseiUnavailable):
            fsei.load(str(tmp_path / "libfsei.so"))
    finally:
        fsei._lib = saved
