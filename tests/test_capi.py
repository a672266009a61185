"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/mcg.h declares; argument validation (host logic, no GPU work) returns
the documented status codes.  Runs without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "mcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mcg_[A-Za-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def mcg():
    from paper_0807_0264_gb300 import mcg as m

    return m


def test_library_exports_every_declared_symbol(mcg):
    declared = header_functions()
    assert len(declared) >= 15
    lib = ctypes.CDLL(mcg.library_path())
    for name in declared:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", mcg.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mcg_[A-Za-z0-9_]+)$", out, flags=re.M))
    assert set(declared) <= exported
    assert set(mcg.EXPORTS) == set(declared)


def test_library_is_built_for_sm_103a(mcg):
    out = subprocess.run(["cuobjdump", "--list-elf", mcg.library_path()], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_version_and_error_codes_without_gpu(mcg):
    lib = mcg.library()
    assert lib.mcg_version() == 10000
    bad = mcg.lattice((3, 4, 4, 4))
    p = mcg.Params().c()
    rc = lib.mcg_fix(ctypes.c_void_p(1), ctypes.c_void_p(2), ctypes.byref(bad), ctypes.byref(p), None, None, None, None)
    assert rc == 2  # MCG_BAD_DIMS
    assert b"even" in lib.mcg_last_error()
    good = mcg.lattice((4, 4, 4, 4))
    rc = lib.mcg_fix(None, ctypes.c_void_p(2), ctypes.byref(good), ctypes.byref(p), None, None, None, None)
    assert rc == 3  # MCG_BAD_ARG
    p.check_every = 0
    rc = lib.mcg_fix(ctypes.c_void_p(1), ctypes.c_void_p(2), ctypes.byref(good), ctypes.byref(p), None, None, None,
                     None)
    assert rc == 3
    zero = mcg.lattice((4, 4, 4, 4), nfields=0)
    assert lib.mcg_plaquette(ctypes.c_void_p(1), None, ctypes.byref(zero), None) == 2
    assert lib.mcg_smear(ctypes.c_void_p(1), ctypes.c_void_p(1), ctypes.byref(good), 0.1, 1.0, 1, None) == 3
    assert lib.mcg_convert(None, 0, ctypes.c_void_p(1), 1, 10, None) == 3
