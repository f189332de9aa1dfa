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
    assert lib.fsei_step_host(None, None, None, None, None, None, ctypes.byref(prm), 1, None,
                              None) == 1
    assert lib.fsei_step_host_join(None, None) == 1
    lib.fsei_grid_destroy(None)


def test_missing_library_fails_loudly(tmp_path):
    saved = fsei._lib
    try:
        fsei._lib = None
        with pytest.raises(fsei.FseiUnavailable):
            fsei.load(str(tmp_path / "libfsei.so"))
    finally:
        fsei._lib = saved


def _header_structs():
    """typedef struct { ... } name; blocks of include/fsei.h: name -> field
    names in declaration order."""
    text = open(os.path.join(ROOT, "include", "fsei.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(\w+)\s*;", text, re.S):
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            # drop the type (first word(s) before the declarators)
            m = re.match(r"(?:const\s+)?\w+\s*(.*)$", decl, re.S)
            for d in m.group(1).split(","):
                fields.append(re.sub(r"[\s*]|\[.*?\]", "", d))
        out[name] = fields
    return out


CTYPES_OF = {"fsei_grid_desc": "GridDesc", "fsei_state": "State",
             "fsei_step_params": "StepParams", "fsei_step_stats": "StepStats",
             "fsei_schedule": "Schedule"}


def test_binding_structs_match_header_fields():
    structs = _header_structs()
    assert set(CTYPES_OF) <= set(structs), structs.keys()
    for cname, pyname in CTYPES_OF.items():
        py = [f for f, _ in getattr(fsei, pyname)._fields_]
        assert py == structs[cname], (cname, py, structs[cname])


def test_binding_struct_layouts_match_c_compiler(tmp_path):
    """sizeof and every field offset of the header's structs, as a C compiler
    lays them out, against the ctypes mirrors of the binding."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = _header_structs()
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "fsei.h"', "int main(void) {"]
    for cname in CTYPES_OF:
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for f in structs[cname]:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True,
                             text=True).stdout.splitlines():
        a, b, v = ln.split()
        got[(a, b)] = int(v)
    for cname, pyname in CTYPES_OF.items():
        cls = getattr(fsei, pyname)
        assert ctypes.sizeof(cls) == got[(cname, "sizeof")], cname
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == got[(cname, f)], (cname, f)


def test_schedule_calls_reject_null_handles(lib):
    s = fsei.Schedule()
    assert lib.fsei_grid_autotune(None, 0, None, ctypes.byref(s)) == 1
    assert lib.fsei_grid_get_schedule(None, ctypes.byref(s)) == 1
    assert lib.fsei_grid_set_schedule(None, ctypes.byref(s)) == 1
    assert lib.fsei_batch_autotune(None, 0, None) == 1


def test_status_names_match_header_enum():
    """The binding's status table is the header's fsei_status enum."""
    text = open(os.path.join(ROOT, "include", "fsei.h")).read()
    body = re.search(r"typedef enum \{(.*?)\} fsei_status;", text, re.S).group(1)
    enum = {int(v): n for n, v in re.findall(r"(FSEI_\w+)\s*=\s*(\d+)", body)}
    assert enum == fsei.STATUS_NAMES


def test_bounds_check_rejects_a_null_handle(lib):
    lib.fsei_grid_check_bounds.argtypes = [ctypes.c_void_p]
    lib.fsei_grid_check_bounds.restype = ctypes.c_int
    assert lib.fsei_grid_check_bounds(None) == 1


def test_poke_guard_rejects_a_null_handle(lib):
    lib.fsei_grid_poke_guard.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int64]
    lib.fsei_grid_poke_guard.restype = ctypes.c_int
    assert lib.fsei_grid_poke_guard(None, 0, 0, 0) == 1
