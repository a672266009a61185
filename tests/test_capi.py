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


def test_library_is_built_for_sm_103a_only(monkeypatch):
    """Every nvcc command of build() (each translation unit and the link)
    targets exactly sm_103a; recorded with nvcc stubbed out, nothing built."""
    import types

    from paper_0807_0264_gb300 import build as b

    cmds = []

    def fake_run(cmd, **kw):
        cmds.append(list(cmd))
        return types.SimpleNamespace(returncode=0, stdout="", stderr="")

    monkeypatch.setattr(b.subprocess, "run", fake_run)
    monkeypatch.setattr(b.os, "makedirs", lambda *a, **k: None)
    monkeypatch.setattr(b.os, "replace", lambda *a, **k: None)
    monkeypatch.setattr(b, "_stale", lambda *a, **k: True)
    b.build(force=True)
    assert len(cmds) == len(b.SOURCES) + 1  # one compile per source, one link
    for cmd in cmds:
        gencodes = [cmd[k + 1] for k, f in enumerate(cmd) if f == "-gencode"]
        assert gencodes == ["arch=compute_103a,code=sm_103a"], cmd
        assert not any(f.startswith(("-arch", "--gpu-architecture", "--gpu-code", "-code")) for f in cmd), cmd



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


def test_argument_validation_of_observables_and_params_without_gpu(mcg):
    """Invalid calls to the Sec. III.A entries and bad parameters are refused
    with MCG_BAD_ARG before any device work, each for its own reason."""
    lib = mcg.library()
    good = mcg.lattice((4, 4, 4, 6))
    one, two = ctypes.c_void_p(1), ctypes.c_void_p(2)

    def refused(rc, why):
        assert rc == 3, rc
        assert why.encode() in lib.mcg_last_error(), lib.mcg_last_error()

    # center decomposition: null inputs, no output requested
    refused(lib.mcg_vortex_remove(None, one, one, None, ctypes.byref(good), None), "null pointer")
    refused(lib.mcg_vortex_remove(one, one, None, None, ctypes.byref(good), None), "no output requested")
    # Wilson loops: R beyond the smallest spatial extent (4), T beyond N_t (6), empty ranges
    W = (ctypes.c_double * 64)()
    for R, T in ((0, 1), (5, 1), (1, 0), (1, 7)):
        refused(lib.mcg_wilson_loops(one, ctypes.byref(good), R, T, W, None), "1 <= Rmax")
    # off-axis: zero vector, a component as long as an extent, T out of range, no vectors
    for vec, T, why in (((0, 0, 0), 1, "path length"), ((4, 0, 0), 1, "smallest spatial extent"),
                        ((0, -4, 1), 1, "smallest spatial extent"), ((1, 1, 0), 7, "Tmax")):
        v = (ctypes.c_int * 3)(*vec)
        refused(lib.mcg_wilson_loops_offaxis(one, ctypes.byref(good), v, 1, T, W, None), why)
    v = (ctypes.c_int * 3)(1, 1, 0)
    refused(lib.mcg_wilson_loops_offaxis(one, ctypes.byref(good), v, 0, 1, W, None), "nvec")
    # parameters: fp64_solve32 in {0, 1}; fp32_overrelax in (0, 2) when an FP32 phase runs
    p = mcg.Params(fp64_solve32=2).c()
    refused(lib.mcg_fix(one, two, ctypes.byref(good), ctypes.byref(p), None, None, None, None), "fp64_solve32")
    for w in (0.0, 2.0, float("nan")):
        p = mcg.Params(fp32_sweeps=10, fp32_overrelax=w).c()
        refused(lib.mcg_fix(one, two, ctypes.byref(good), ctypes.byref(p), None, None, None, None), "overrelax")


def test_anneal_argument_validation_without_gpu(mcg):
    """mcg_anneal refuses bad arguments with MCG_BAD_ARG before device work."""
    lib = mcg.library()
    one, two = ctypes.c_void_p(1), ctypes.c_void_p(1 << 40)
    T = (ctypes.c_double * 3)(1.0, 0.5, 0.1)

    def refused(lat, T_, n, first, nhit, eps, why, U=one, G=two):
        rc = lib.mcg_anneal(U, G, ctypes.byref(lat), T_, n, first, nhit, eps, 7, None, None)
        assert rc == 3, rc
        assert why.encode() in lib.mcg_last_error(), lib.mcg_last_error()

    f64 = mcg.lattice((4, 4, 4, 6))
    refused(mcg.lattice((4, 4, 4, 6), 1, mcg.F32), T, 3, 0, 1, 0.3, "FP64")
    refused(mcg.lattice((4, 4, 4, 6), 70000), T, 3, 0, 1, 0.3, "65535")
    refused(f64, None, 3, 0, 1, 0.3, "null pointer")
    refused(f64, T, 3, 0, 1, 0.3, "null pointer", G=None)
    refused(f64, T, -1, 0, 1, 0.3, ">= 0")
    refused(f64, T, 3, -2, 1, 0.3, ">= 0")
    refused(f64, T, 3, 0, 0, 0.3, "nhit")
    for eps in (0.0, 0.51, float("nan")):
        refused(f64, T, 3, 0, 2, eps, "eps")
    for bad in (0.0, -1.0, float("nan")):
        Tb = (ctypes.c_double * 3)(1.0, bad, 0.1)
        refused(f64, Tb, 3, 0, 2, 0.3, "temperature")
    refused(f64, T, 3, 0, 2, 0.3, "overlap", U=one, G=ctypes.c_void_p(1 + 4096))


def test_anneal_schedule_is_geometric(mcg):
    T = mcg.anneal_schedule(2.0, 0.02, 5)
    assert len(T) == 5 and T[0] == 2.0 and abs(T[-1] - 0.02) < 1e-15
    r = [T[k + 1] / T[k] for k in range(4)]
    assert max(r) - min(r) < 1e-14 and abs(r[0] - 0.1 ** 0.5) < 1e-14
    assert mcg.anneal_schedule(3.0, 0.1, 1) == [3.0]
    assert mcg.anneal_schedule(3.0, 0.1, 0) == []


def test_slab_phase_stats_and_bounds_validation_without_gpu(mcg):
    """The slab half-sweep, the phase statistics, the double-float flag and the
    lattice bounds are checked on the host before any device work."""
    lib = mcg.library()
    one, two = ctypes.c_void_p(1), ctypes.c_void_p(1 << 40)
    good = mcg.lattice((4, 4, 4, 6))

    def code(rc, want, why):
        assert rc == want, rc
        assert why.encode() in lib.mcg_last_error(), lib.mcg_last_error()

    for t_lo, t_hi in ((0, 0), (-1, 3), (2, 7), (4, 3)):
        code(lib.mcg_halfsweep_slab(one, two, ctypes.byref(good), 0, t_lo, t_hi, None, None), 3, "t_lo")
    code(lib.mcg_halfsweep_slab(one, two, ctypes.byref(good), 2, 0, 6, None, None), 3, "parity")
    code(lib.mcg_halfsweep_slab(one, two, ctypes.byref(mcg.lattice((4, 4, 4, 6), 1, mcg.F32)), 0, 0, 6, None, None),
         3, "FP64")
    code(lib.mcg_halfsweep_slab(one, two, ctypes.byref(mcg.lattice((4, 4, 4, 6), 2)), 0, 0, 6, None, None), 3,
         "FP64")
    code(lib.mcg_halfsweep_slab(None, two, ctypes.byref(good), 0, 0, 6, None, None), 3, "null")
    code(lib.mcg_phase_stats(None, None, 0), 3, "null")
    ms = (ctypes.c_double * 2)()
    su = (ctypes.c_longlong * 2)()
    assert lib.mcg_phase_stats(ms, su, 1) == 0 and ms[0] >= 0 and su[1] >= 0
    p = mcg.Params(fp64_df=2).c()
    code(lib.mcg_fix(one, two, ctypes.byref(good), ctypes.byref(p), None, None, None, None), 3, "fp64_df")
    # extents are bounded before the volume is formed: no int input overflows
    for dims in ((1 << 16, 2, 2, 2), (2, 2, 2, (1 << 31) - 1 - 1)):
        huge = mcg.lattice(dims)
        code(lib.mcg_plaquette_static(one, one, ctypes.byref(huge), None), 2, "")
        code(lib.mcg_plaquette(one, None, ctypes.byref(huge), None), 2, "")
    code(lib.mcg_plaquette(one, None, ctypes.byref(mcg.lattice((4, 4, 4, 4), 1 << 21)), None), 2, "nfields")


def test_regular_build_reports_no_index_checks(mcg):
    """mcg_bounds_violations answers -1 in a build without -DMCG_CHECK, with
    no device call."""
    assert mcg.library().mcg_bounds_violations(0) == -1


def test_slab_face_validation_without_gpu(mcg):
    """The slab face copy checks layer, parity, direction, field count,
    pointers and overlap on the host before any device work."""
    lib = mcg.library()
    U, buf = ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 40)
    good = mcg.lattice((4, 4, 4, 6))

    def code(rc, want, why):
        assert rc == want, rc
        assert why.encode() in lib.mcg_last_error(), lib.mcg_last_error()

    for t in (-1, 6):
        code(lib.mcg_slab_face(U, buf, ctypes.byref(good), t, 0, 0, None), 3, "N_t")
    code(lib.mcg_slab_face(U, buf, ctypes.byref(good), 0, 2, 0, None), 3, "parity")
    code(lib.mcg_slab_face(U, buf, ctypes.byref(good), 0, 0, 2, None), 3, "to_field")
    code(lib.mcg_slab_face(U, buf, ctypes.byref(mcg.lattice((4, 4, 4, 6), 2)), 0, 0, 0, None), 3, "one field")
    code(lib.mcg_slab_face(None, buf, ctypes.byref(good), 0, 0, 0, None), 3, "null")
    code(lib.mcg_slab_face(U, None, ctypes.byref(good), 0, 0, 0, None), 3, "null")
    # a buffer inside the field (FP64 links of 4^3 x 6: 72 x 192 x 16 bytes)
    inside = ctypes.c_void_p((1 << 20) + 4096)
    code(lib.mcg_slab_face(U, inside, ctypes.byref(good), 0, 0, 0, None), 3, "overlaps")
    code(lib.mcg_slab_face(U, buf, ctypes.byref(mcg.lattice((4, 3, 4, 6))), 0, 0, 0, None), 2, "")


def test_restart_and_finish_parameters_are_validated_without_gpu(mcg):
    lib = mcg.library()
    one, two = ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 40)
    good = mcg.lattice((4, 4, 4, 6))
    for field, value, why in (("fp32_restart", -1, "fp32_restart"), ("fp32_restart_domega", -0.1, "domega"),
                              ("fp32_restart_domega", 2.0, "domega"), ("fp32_restart_random", 2, "random"),
                              ("fp32_restart_creep", -5, "creep"), ("fp32_plain_finish", 3, "plain_finish")):
        p = mcg.Params(fp32_sweeps=10)
        setattr(p, field, value)
        cp = p.c()
        assert lib.mcg_fix(one, two, ctypes.byref(good), ctypes.byref(cp), None, None, None, None) == 3
        assert why.encode() in lib.mcg_last_error(), lib.mcg_last_error()


def test_local_solve_validation_without_gpu(mcg):
    """The batched local solve checks its count, precision and pointers on the
    host; n = 0 is a no-op that touches no device memory."""
    lib = mcg.library()
    one = ctypes.c_void_p(1 << 20)

    def code(rc, want, why):
        assert rc == want, rc
        assert why.encode() in lib.mcg_last_error(), lib.mcg_last_error()

    code(lib.mcg_local_solve(one, one, one, None, -1, mcg.F64, None), 3, "n must be")
    code(lib.mcg_local_solve(one, one, one, None, 4, 2, None), 3, "precision")
    code(lib.mcg_local_solve(None, one, one, None, 4, mcg.F32, None), 3, "null")
    code(lib.mcg_local_solve(one, one, None, None, 4, mcg.F64, None), 3, "null")
    assert lib.mcg_local_solve(None, None, None, None, 0, mcg.F32, None) == 0
