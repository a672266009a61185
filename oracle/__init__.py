"""FP64 CPU oracle for MCG fixing with stout / over-improved stout preconditioning.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are its only users.  The product path never imports it.

The arithmetic lives in `mcg_oracle.c` (plain C99, FP64, optional OpenMP);
this module compiles it with gcc on first use and exposes numpy-array
wrappers.  Arrays use the canonical host layout of `synth.py`:
U (V, 4, 3, 3) complex128, Omega (V, 3, 3) complex128, site index
x + Nx*(y + Ny*(z + Nz*t)).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcg_oracle.c")
_LIB = os.path.join(_HERE, "libmcg_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc -O2 -fopenmp)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            D = ctypes.c_double
            I = ctypes.c_int
            L = ctypes.c_long
            lib.orc_functional_R.argtypes = [P, P]
            lib.orc_functional_R.restype = D
            lib.orc_plaquette.argtypes = [P, P]
            lib.orc_plaquette.restype = D
            lib.orc_apply_gauge.argtypes = [P, P, P]
            lib.orc_reunitarise_field.argtypes = [L, P]
            lib.orc_compose_gauge.argtypes = [L, P, P, P]
            lib.orc_trs_solve.argtypes = [P, P, P]
            lib.orc_trs_solve.restype = I
            lib.orc_halfsweep.argtypes = [P, P, P, I, D]
            lib.orc_halfsweep.restype = L
            lib.orc_fix.argtypes = [P, P, P, D, I, I, D, P, P, P]
            lib.orc_halfsweep_slab.argtypes = [P, P, P, I, D, I, I, I]
            lib.orc_halfsweep_slab.restype = L
            U64 = ctypes.c_uint64
            lib.orc_philox4x64.argtypes = [P, P, P]
            lib.orc_anneal_halfsweep.argtypes = [P, P, P, I, D, L, I, D, U64, U64]
            lib.orc_anneal_halfsweep.restype = L
            lib.orc_anneal.argtypes = [P, P, P, P, I, L, I, D, U64, U64]
            lib.orc_anneal.restype = L
            lib.orc_fix.restype = I
            lib.orc_expm.argtypes = [P, P]
            lib.orc_smear_step.argtypes = [P, P, P, D, D]
            lib.orc_smear.argtypes = [P, P, P, D, D, I]
            lib.orc_center_project.argtypes = [P, P, P]
            lib.orc_vortex_count.argtypes = [P, P, P]
            lib.orc_vortex_count.restype = ctypes.c_longlong
            lib.orc_grad_R.argtypes = [P, P, P]
            lib.orc_generators.argtypes = [P]
            lib.orc_expm_frechet.argtypes = [P, P, P]
            lib.orc_staple_sum_paths.argtypes = [P, P, L, I, D, D, P]
            lib.orc_staple_sum.argtypes = [P, P, L, I, D, D, P]
            lib.orc_smear_step_backward.argtypes = [P, P, P, P, D, D]
            lib.orc_functional_matrix_grad.argtypes = [P, P, P]
            lib.orc_vortex_remove.argtypes = [P, P, P, P]
            lib.orc_center_links.argtypes = [P, P, P]
            lib.orc_wilson_loops.argtypes = [P, P, I, I, P]
            lib.orc_wilson_loops_offaxis.argtypes = [P, P, P, I, I, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(dims) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int32))


def _cfield(U) -> np.ndarray:
    return np.ascontiguousarray(U, dtype=np.complex128)


def set_threads(n: int) -> None:
    """OpenMP thread count for subsequent calls (libgomp honours the env var
    only at start-up, so this goes through omp_set_num_threads)."""
    gomp = ctypes.CDLL("libgomp.so.1")
    gomp.omp_set_num_threads(int(n))


def functional_R(dims, U) -> float:
    U = _cfield(U)
    return _load().orc_functional_R(_p(_dims(dims)), _p(U))


def functional_V(dims, U) -> float:
    vol = int(np.prod(dims))
    return functional_R(dims, U) / (36.0 * vol)


def plaquette(dims, U) -> float:
    U = _cfield(U)
    return _load().orc_plaquette(_p(_dims(dims)), _p(U))


def apply_gauge(dims, U, G) -> np.ndarray:
    out = _cfield(U).copy()
    G = _cfield(G)
    _load().orc_apply_gauge(_p(_dims(dims)), _p(out), _p(G))
    return out


def reunitarise(M) -> np.ndarray:
    out = _cfield(M).copy()
    _load().orc_reunitarise_field(out.size // 9, _p(out))
    return out


def compose_gauge(Gb, Ga) -> np.ndarray:
    Gb = _cfield(Gb)
    Ga = _cfield(Ga)
    out = np.empty_like(Ga)
    _load().orc_compose_gauge(Ga.size // 9, _p(Gb), _p(Ga), _p(out))
    return out


def trs_solve(A, b):
    """Maximise a^T A a + 2 b.a on |a| = 1.  Returns (a, hard_case)."""
    A = np.ascontiguousarray(A, dtype=np.float64).reshape(4, 4)
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(4)
    a = np.zeros(4)
    hard = _load().orc_trs_solve(_p(A), _p(b), _p(a))
    return a, bool(hard)


def halfsweep(dims, U, G, parity: int, omega: float = 1.0):
    """One checkerboard half-sweep; returns (U', G', hard_case_count)."""
    U = _cfield(U).copy()
    G = _cfield(G).copy()
    hard = _load().orc_halfsweep(_p(_dims(dims)), _p(U), _p(G), int(parity), float(omega))
    return U, G, int(hard)


def halfsweep_slab(dims, U, G, parity: int, t_lo: int, t_hi: int, t_offset: int = 0, omega: float = 1.0):
    """Half-sweep of the sites with t_lo <= t < t_hi of the local array U
    (a slab of a larger lattice plus ghost layers) whose whole-lattice parity
    (x+y+z+t+t_offset) mod 2 is `parity`; in place.  Returns the number of
    hard-case solves."""
    assert U.flags["C_CONTIGUOUS"] and U.dtype == np.complex128
    assert G.flags["C_CONTIGUOUS"] and G.dtype == np.complex128
    return int(_load().orc_halfsweep_slab(_p(_dims(dims)), _p(U), _p(G), int(parity), float(omega), int(t_lo),
                                          int(t_hi), int(t_offset)))


def fix(dims, U, G=None, tol: float = 1e-10, max_sweeps: int = 2000, reunit_every: int = 50, omega: float = 1.0):
    """MCG relaxation.  Returns dict(U, G, R_hist, sweeps, converged, hard)."""
    U = _cfield(U).copy()
    vol = U.shape[0]
    if G is None:
        G = np.zeros((vol, 3, 3), np.complex128)
        G[:, 0, 0] = G[:, 1, 1] = G[:, 2, 2] = 1
    G = _cfield(G).copy()
    R_hist = np.zeros(max_sweeps + 1)
    sweeps = ctypes.c_int(0)
    hard = ctypes.c_long(0)
    rc = _load().orc_fix(_p(_dims(dims)), _p(U), _p(G), float(tol), int(max_sweeps), int(reunit_every),
                         float(omega), _p(R_hist), ctypes.byref(sweeps), ctypes.byref(hard))
    n = sweeps.value
    return dict(U=U, G=G, R_hist=R_hist[: n + 1], sweeps=n, converged=(rc == 0), hard=int(hard.value))


def philox4x64(counter, key) -> np.ndarray:
    """Philox4x64-10 block for a 4-word counter and 2-word key (uint64)."""
    c = np.ascontiguousarray(counter, dtype=np.uint64).reshape(4)
    k = np.ascontiguousarray(key, dtype=np.uint64).reshape(2)
    out = np.zeros(4, np.uint64)
    _load().orc_philox4x64(_p(c), _p(k), _p(out))
    return out


def anneal_halfsweep(dims, U, G, parity: int, T: float, sweep: int, nhit: int, eps: float, seed: int,
                     field: int = 0):
    """One annealing half-sweep; returns (U', G', accepted hits)."""
    U = _cfield(U).copy()
    G = _cfield(G).copy()
    acc = _load().orc_anneal_halfsweep(_p(_dims(dims)), _p(U), _p(G), int(parity), float(T), int(sweep), int(nhit),
                                       float(eps), int(seed), int(field))
    return U, G, int(acc)


def anneal(dims, U, G, T, nhit: int, eps: float, seed: int, first_sweep: int = 0, field: int = 0):
    """Simulated annealing with temperatures T[k] (one per sweep), then
    re-unitarisation.  Returns (U', G', accepted hits)."""
    U = _cfield(U).copy()
    G = _cfield(G).copy()
    T = np.ascontiguousarray(T, dtype=np.float64).reshape(-1)
    acc = _load().orc_anneal(_p(_dims(dims)), _p(U), _p(G), _p(T), int(T.size), int(first_sweep), int(nhit),
                             float(eps), int(seed), int(field))
    return U, G, int(acc)


def expm(X) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.complex128).reshape(3, 3)
    E = np.zeros((3, 3), np.complex128)
    _load().orc_expm(_p(X), _p(E))
    return E


def smear(dims, U, rho: float, eps: float, nsteps: int) -> np.ndarray:
    """nsteps of stout (eps = 1) or over-improved stout smearing."""
    U = _cfield(U)
    out = np.empty_like(U)
    _load().orc_smear(_p(_dims(dims)), _p(U), _p(out), float(rho), float(eps), int(nsteps))
    return out


def center_project(dims, U) -> np.ndarray:
    """Center sector m in {-1, 0, 1} per link, shape (V, 4) int8."""
    U = _cfield(U)
    m = np.zeros((U.shape[0], 4), np.int8)
    _load().orc_center_project(_p(_dims(dims)), _p(U), _p(m))
    return m


def vortex_count(dims, m):
    """(total, per_plane[6]) P-vortex plaquettes from center sectors m."""
    m = np.ascontiguousarray(m, dtype=np.int8)
    per = np.zeros(6, np.int64)
    tot = _load().orc_vortex_count(_p(_dims(dims)), _p(m), _p(per))
    return int(tot), per


def grad_R(dims, U) -> np.ndarray:
    """dR/d eps_a(x) for Omega(x) -> exp(i eps T_a) Omega(x); shape (V, 8)."""
    U = _cfield(U)
    out = np.zeros((U.shape[0], 8))
    _load().orc_grad_R(_p(_dims(dims)), _p(U), _p(out))
    return out


def generators() -> np.ndarray:
    """The oracle's T_a = lambda_a / 2, shape (8, 3, 3)."""
    T = np.zeros((8, 3, 3), np.complex128)
    _load().orc_generators(_p(T))
    return T


def precondition_and_fix(dims, U, rho: float, eps: float, nsmear: int, tol: float = 1e-10,
                         max_sweeps: int = 2000, reunit_every: int = 50):
    """The preconditioning pipeline of Sec. II.B, step by step:
    smear the field; MCG-fix the smeared field keeping the total transform
    Omega_1; apply Omega_1 to the original (unsmeared) field; MCG-fix that
    preconditioned field.  With nsmear = 0 the first fix is skipped (no
    preconditioning).  Returns a dict of the stages' results."""
    U = _cfield(U)
    vol = U.shape[0]
    out = {}
    if nsmear > 0:
        S = smear(dims, U, rho, eps, nsmear)
        r1 = fix(dims, S, None, tol, max_sweeps, reunit_every)
        out["smeared"] = r1
        G1 = reunitarise(r1["G"])
        Up = apply_gauge(dims, U, G1)
    else:
        G1 = np.zeros((vol, 3, 3), np.complex128)
        G1[:, 0, 0] = G1[:, 1, 1] = G1[:, 2, 2] = 1
        Up = U.copy()
    r2 = fix(dims, Up, None, tol, max_sweeps, reunit_every)
    out["fixed"] = r2
    m = center_project(dims, r2["U"])
    tot, per = vortex_count(dims, m)
    out["m"] = m
    out["vortices"] = tot
    out["vortex_density"] = tot / (6.0 * vol)
    out["G_total"] = compose_gauge(r2["G"], G1)
    return out


def expm_frechet(X, A) -> np.ndarray:
    """L(X, A) = d/dt exp(X + tA) at t = 0 for 3x3 complex X, A."""
    X = np.ascontiguousarray(X, dtype=np.complex128).reshape(3, 3)
    A = np.ascontiguousarray(A, dtype=np.complex128).reshape(3, 3)
    L = np.zeros((3, 3), np.complex128)
    _load().orc_expm_frechet(_p(X), _p(A), _p(L))
    return L


def staple_sum(dims, U, x: int, mu: int, cp: float, cr: float, from_paths: bool = False) -> np.ndarray:
    U = _cfield(U)
    C = np.zeros((3, 3), np.complex128)
    fn = _load().orc_staple_sum_paths if from_paths else _load().orc_staple_sum
    fn(_p(_dims(dims)), _p(U), int(x), int(mu), float(cp), float(cr), _p(C))
    return C


def functional_matrix_grad(dims, U) -> np.ndarray:
    """dR/dRe U + i dR/dIm U = 2 tr(U) 1 per link, shape (V, 4, 3, 3)."""
    U = _cfield(U)
    G = np.zeros_like(U)
    _load().orc_functional_matrix_grad(_p(_dims(dims)), _p(U), _p(G))
    return G


def smear_step_backward(dims, U, Gout, rho: float, eps: float) -> np.ndarray:
    """Gradient w.r.t. the input of one smearing step, given the gradient
    Gout (= dL/dRe U' + i dL/dIm U') w.r.t. its output."""
    U = _cfield(U)
    Gout = _cfield(Gout)
    Gin = np.zeros_like(U)
    _load().orc_smear_step_backward(_p(_dims(dims)), _p(U), _p(Gout), _p(Gin), float(rho), float(eps))
    return Gin


def smear_backward(dims, U, Gout, rho: float, eps: float, nsteps: int) -> np.ndarray:
    """Gradient w.r.t. U of a loss of smear(U, rho, eps, nsteps), given its
    gradient Gout w.r.t. the smeared field; the intermediate fields are
    recomputed (stored) by forward smearing."""
    fields = [_cfield(U)]
    for _ in range(nsteps - 1):
        fields.append(smear(dims, fields[-1], rho, eps, 1))
    G = _cfield(Gout)
    for k in range(nsteps - 1, -1, -1):
        G = smear_step_backward(dims, fields[k], G, rho, eps)
    return G


def vortex_remove(dims, U, m) -> np.ndarray:
    """Vortex-removed field U' = Z^dag U (Sec. III.A) for center sectors m (V, 4)."""
    U = _cfield(U)
    m = np.ascontiguousarray(m, dtype=np.int8)
    out = np.empty_like(U)
    _load().orc_vortex_remove(_p(_dims(dims)), _p(U), _p(m), _p(out))
    return out


def center_links(dims, m) -> np.ndarray:
    """The vortex-only field Z = exp(2 pi i m / 3) * 1 (Sec. III.A), shape (V, 4, 3, 3)."""
    m = np.ascontiguousarray(m, dtype=np.int8)
    out = np.empty((m.shape[0], 4, 3, 3), np.complex128)
    _load().orc_center_links(_p(_dims(dims)), _p(m), _p(out))
    return out


def wilson_loops(dims, U, Rmax: int, Tmax: int) -> np.ndarray:
    """Planar Wilson loops W(R, T) (Sec. III.A), R spatial (averaged over x, y, z),
    T along t, averaged over all translations; shape (Rmax, Tmax)."""
    U = _cfield(U)
    out = np.zeros(Rmax * Tmax)
    _load().orc_wilson_loops(_p(_dims(dims)), _p(U), int(Rmax), int(Tmax), _p(out))
    return out.reshape(Rmax, Tmax)


def wilson_loops_offaxis(dims, U, vectors, Tmax: int) -> np.ndarray:
    """Wilson loops with spatial side r (any integer 3-vector, off-axis
    allowed) and temporal side T (Sec. III.A), averaged over all translations
    and the distinct cubic images of r; shape (len(vectors), Tmax)."""
    U = _cfield(U)
    v = np.ascontiguousarray(np.asarray(vectors, dtype=np.int32).reshape(-1, 3))
    out = np.zeros(v.shape[0] * Tmax)
    _load().orc_wilson_loops_offaxis(_p(_dims(dims)), _p(U), _p(v), int(v.shape[0]), int(Tmax), _p(out))
    return out.reshape(v.shape[0], Tmax)
