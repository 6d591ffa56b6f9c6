"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/bsc.h (no GPU needed: no compute call is made)."""
import ctypes as ct
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bsc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bsc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2506_18867_gb300 import build
    return build.build()


def test_header_and_binding_agree():
    from paper_2506_18867_gb300 import bsc
    assert sorted(bsc.EXPORTS) == _declared()


def test_library_exports_every_declared_symbol(libpath):
    lib = ct.CDLL(libpath)
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (bsc_\w+)", out))
    assert set(_declared()) <= exported


def test_library_is_built_for_sm_103a(libpath):
    out = subprocess.run(["cuobjdump", "--list-elf", libpath], capture_output=True, text=True).stdout
    assert "sm_103a" in out or "sm_103" in out


def test_create_without_gpu_fails_cleanly(libpath):
    """On a host without a GPU bsc_create must return an error, not abort."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2506_18867_gb300 import bsc
    lib = bsc.load(libpath)
    grid = bsc.KnotGrid(5, 5, None, None)
    rest = (ct.c_double * 50)()
    mat = bsc.Material(1, 1, 1, 1, 1)
    opt = bsc.Options()
    h = ct.c_void_p()
    st = lib.bsc_create(ct.byref(grid), rest, ct.byref(mat), None, ct.byref(opt), None, ct.byref(h))
    assert st != bsc.OK and not h.value
    assert lib.bsc_last_error(None)


def test_create_rejects_bad_arguments(libpath):
    from paper_2506_18867_gb300 import bsc
    lib = bsc.load(libpath)
    rest = (ct.c_double * 32)()
    mat = bsc.Material(1, 1, 1, 1, 1)
    opt = bsc.Options()
    h = ct.c_void_p()
    grid = bsc.KnotGrid(4, 4, None, None)  # fewer than 5 control points per axis
    assert lib.bsc_create(ct.byref(grid), rest, ct.byref(mat), None, ct.byref(opt), None,
                          ct.byref(h)) == bsc.ERR_INVALID_ARG
    assert b"5" in lib.bsc_last_error(None)
    grid = bsc.KnotGrid(5, 5, None, None)
    rest = (ct.c_double * 50)()
    bad_knots = (ct.c_double * 8)(0, 0, 0, 1, 2, 4, 4, 4)
    grid_k = bsc.KnotGrid(5, 5, bad_knots, None)
    assert lib.bsc_create(ct.byref(grid_k), rest, ct.byref(mat), None, ct.byref(opt), None,
                          ct.byref(h)) == bsc.ERR_INVALID_ARG
    pins = (ct.c_int32 * 1)(99)
    opt2 = bsc.Options(0, 0.01, (ct.c_double * 3)(0, 0, 0), pins, 1, 1, 1e-8, 100, 30)
    assert lib.bsc_create(ct.byref(grid), rest, ct.byref(mat), None, ct.byref(opt2), None,
                          ct.byref(h)) == bsc.ERR_INVALID_ARG
    assert b"pinned" in lib.bsc_last_error(None)
    nanrest = (ct.c_double * 50)(*([float("nan")] * 50))
    assert lib.bsc_create(ct.byref(grid), nanrest, ct.byref(mat), None, ct.byref(opt), None,
                          ct.byref(h)) == bsc.ERR_INVALID_ARG
