"""Thin Python binding of libmcg (include/mcg.h) over ctypes.

Every function here marshals arguments and calls the C-ABI entry point of the
same name; all computation runs in the CUDA kernels of libmcg.so.  PyTorch
provides device memory (tensors) and the current CUDA stream.  There is no CPU
fallback: if the library is missing, importing this module builds it with
nvcc, and if that fails the import raises.

Tensor conventions (device, even/odd SoA, see include/mcg.h):
    links  U: float64 / float32 tensor (nfields, 4, 2, 9, Vh, 2)  [mu, parity, entry, site, re/im]
    gauge  G: float64 / float32 tensor (nfields, 2, 9, Vh, 2)
    center Z: int8 tensor (nfields, 4, 2, Vh)
    canonical links:  complex128 tensor (nfields, V, 4, 3, 3)
    canonical gauge:  complex128 tensor (nfields, V, 3, 3)
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import torch

from . import build as _build

F64, F32 = 0, 1
OK, NOT_CONVERGED = 0, 1
_STATUS = {0: "MCG_OK", 1: "MCG_NOT_CONVERGED", 2: "MCG_BAD_DIMS", 3: "MCG_BAD_ARG", 4: "MCG_BAD_INPUT",
           5: "MCG_CUDA_ERROR"}


class MCGError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn} -> {_STATUS.get(code, code)}: {msg}")
        self.code = code


class mcg_lattice(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("nfields", ctypes.c_int), ("precision", ctypes.c_int)]


class mcg_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_sweeps", ctypes.c_int), ("check_every", ctypes.c_int),
                ("reunit_every", ctypes.c_int), ("fp32_sweeps", ctypes.c_int), ("fp32_tol", ctypes.c_double),
                ("fp32_window", ctypes.c_int), ("fp32_overrelax", ctypes.c_double),
                ("fp64_solve32", ctypes.c_int), ("fp64_df", ctypes.c_int), ("fp32_restart", ctypes.c_int),
                ("fp32_restart_domega", ctypes.c_double), ("fp32_restart_random", ctypes.c_int),
                ("fp32_restart_creep", ctypes.c_int), ("fp32_plain_finish", ctypes.c_int)]


class mcg_field(ctypes.Structure):
    _fields_ = [("U", ctypes.c_void_p), ("G", ctypes.c_void_p), ("dims", ctypes.c_int * 4)]


class mcg_precond_result(ctypes.Structure):
    _fields_ = [("V_smeared", ctypes.c_double), ("V_fixed", ctypes.c_double), ("plaquette_in", ctypes.c_double),
                ("plaquette_out", ctypes.c_double), ("vortices", ctypes.c_longlong),
                ("vortex_density", ctypes.c_double), ("sweeps_smeared", ctypes.c_int),
                ("sweeps_fixed", ctypes.c_int), ("sweeps_fp32", ctypes.c_int), ("status", ctypes.c_int),
                ("fp32_restarts", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _load() -> ctypes.CDLL:
    # MCG_LIBRARY: an explicit libmcg build (e.g. the index-checking one)
    path = os.environ.get("MCG_LIBRARY") or _build.LIB
    if path == _build.LIB and not os.path.exists(path):
        _build.build()
    lib = ctypes.CDLL(path)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    L = ctypes.POINTER(mcg_lattice)
    PR = ctypes.POINTER(mcg_params)
    sig = {
        "mcg_version": ([], I),
        "mcg_last_error": ([], ctypes.c_char_p),
        "mcg_release": ([], I),
        "mcg_pack_links": ([P, P, L, P], I),
        "mcg_unpack_links": ([P, P, L, P], I),
        "mcg_pack_gauge": ([P, P, L, P], I),
        "mcg_unpack_gauge": ([P, P, L, P], I),
        "mcg_unpack_center": ([P, P, L, P], I),
        "mcg_convert": ([P, I, P, I, S, P], I),
        "mcg_set_identity_gauge": ([P, L, P], I),
        "mcg_plaquette": ([P, P, L, P], I),
        "mcg_functional": ([P, P, L, P], I),
        "mcg_apply_gauge": ([P, P, L, P], I),
        "mcg_reunitarise": ([P, I, L, P], I),
        "mcg_smear": ([P, P, L, D, D, I, P], I),
        "mcg_fix": ([P, P, L, PR, P, P, P, P], I),
        "mcg_anneal": ([P, P, L, P, I, ctypes.c_longlong, I, D, ctypes.c_ulonglong, P, P], I),
        "mcg_local_solve": ([P, P, P, P, I, I, P], I),
        "mcg_random_gauge": ([P, L, ctypes.c_ulonglong, ctypes.c_ulonglong, P], I),
        "mcg_center_project": ([P, P, P, L, P], I),
        "mcg_vortex_remove": ([P, P, P, P, L, P], I),
        "mcg_wilson_loops": ([P, L, I, I, P, P], I),
        "mcg_wilson_loops_offaxis": ([P, L, P, I, I, P, P], I),
        "mcg_precondition_fix": ([P, P, P, L, PR, D, D, I, I, ctypes.POINTER(mcg_precond_result), P], I),
        "mcg_precondition_levels": ([P, P, P, P, L, PR, D, D, ctypes.POINTER(ctypes.c_int), I, I,
                                     ctypes.POINTER(mcg_precond_result), P], I),
        "mcg_time_halfsweep": ([P, P, L, I, I, I, ctypes.POINTER(ctypes.c_float), P], I),
        "mcg_kernel_launches": ([], ctypes.c_longlong),
        "mcg_halfsweep_slab": ([P, P, L, I, I, I, P, P], I),
        "mcg_slab_face": ([P, P, L, I, I, I, P], I),
        "mcg_bounds_violations": ([I], ctypes.c_longlong),
        "mcg_probe_peaks": ([ctypes.POINTER(ctypes.c_double), P], I),
        "mcg_phase_stats": ([ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong), I], I),
        "mcg_plaquette_static": ([P, P, L, P], I),
        "mcg_set_sweep_block": ([I, I], I),
        "mcg_smear_backward_step": ([P, P, P, L, D, D, P], I),
        "mcg_functional_matrix_grad": ([P, P, L, P], I),
        "mcg_grad_R": ([P, P, L, P], I),
        "mcg_ascent_step": ([P, P, P, D, L, P], I),
        "mcg_fix_batch": ([ctypes.POINTER(mcg_field), I, I, PR, P, P, P], I),
        "mcg_gribov_search": ([ctypes.POINTER(mcg_field), I, ctypes.POINTER(ctypes.c_int), I, I, PR, P, P, P, P, P],
                              I),
        "mcg_get_sweep_block": ([I], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()

#: every entry point include/mcg.h declares (checked by the test suite)
EXPORTS = ("mcg_version", "mcg_last_error", "mcg_release", "mcg_pack_links", "mcg_unpack_links", "mcg_pack_gauge",
           "mcg_unpack_gauge", "mcg_unpack_center", "mcg_convert", "mcg_set_identity_gauge", "mcg_plaquette",
           "mcg_functional", "mcg_apply_gauge", "mcg_reunitarise", "mcg_smear", "mcg_fix", "mcg_center_project",
           "mcg_precondition_fix", "mcg_precondition_levels", "mcg_time_halfsweep", "mcg_kernel_launches",
           "mcg_plaquette_static", "mcg_set_sweep_block", "mcg_get_sweep_block", "mcg_fix_batch",
           "mcg_gribov_search", "mcg_smear_backward_step", "mcg_functional_matrix_grad", "mcg_grad_R",
           "mcg_ascent_step", "mcg_vortex_remove", "mcg_wilson_loops",
           "mcg_wilson_loops_offaxis", "mcg_anneal", "mcg_phase_stats",
           "mcg_halfsweep_slab", "mcg_slab_face", "mcg_bounds_violations", "mcg_probe_peaks", "mcg_local_solve",
           "mcg_random_gauge")
#: seed of the random gauge copies of Params.fp32_restart_random
RESTART_SEED = 0x4D434752


def library() -> ctypes.CDLL:
    return _lib


def library_path() -> str:
    return _build.LIB


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Params:
    """mcg_params: stop threshold on dV_U and the sweep schedule."""
    tol: float = 1e-10
    max_sweeps: int = 2000
    check_every: int = 20
    reunit_every: int = 50
    fp32_sweeps: int = 0
    fp32_tol: float = 1e-10
    fp32_window: int = 25
    fp32_overrelax: float = 1.0
    fp64_solve32: int = 0
    fp64_df: int = 0
    fp32_restart: int = 0
    fp32_restart_domega: float = 0.0
    fp32_restart_random: int = 0
    fp32_restart_creep: int = 0
    fp32_plain_finish: int = 0

    def c(self) -> mcg_params:
        return mcg_params(self.tol, self.max_sweeps, self.check_every, self.reunit_every, self.fp32_sweeps,
                          self.fp32_tol, self.fp32_window, self.fp32_overrelax,
                          int(self.fp64_solve32), int(self.fp64_df), int(self.fp32_restart),
                          float(self.fp32_restart_domega), int(self.fp32_restart_random),
                          int(self.fp32_restart_creep), int(self.fp32_plain_finish))


def lattice(dims, nfields: int = 1, precision: int = F64) -> mcg_lattice:
    lat = mcg_lattice()
    for k in range(4):
        lat.dims[k] = int(dims[k])
    lat.nfields = int(nfields)
    lat.precision = int(precision)
    return lat


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _check(fn: str, rc: int, allow=(OK,)) -> int:
    if rc not in allow:
        raise MCGError(fn, rc, _lib.mcg_last_error().decode())
    return rc


def _real_dtype(precision: int):
    return torch.float64 if precision == F64 else torch.float32


def vh_of(dims) -> int:
    v = 1
    for d in dims:
        v *= int(d)
    return v // 2


def empty_links(dims, nfields=1, precision=F64, device="cuda"):
    return torch.empty((nfields, 4, 2, 9, vh_of(dims), 2), dtype=_real_dtype(precision), device=device)


def empty_gauge(dims, nfields=1, precision=F64, device="cuda"):
    return torch.empty((nfields, 2, 9, vh_of(dims), 2), dtype=_real_dtype(precision), device=device)


def empty_face(dims, precision=F64, device="cuda"):
    """Buffer of one slab face (mcg_slab_face): (9, Nx*Ny*Nz/2, 2) reals."""
    return torch.empty((9, int(dims[0]) * int(dims[1]) * int(dims[2]) // 2, 2), dtype=_real_dtype(precision),
                       device=device)


def precision_of(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"field tensor must be float64 or float32, got {t.dtype}")


def _need_cuda(*ts):
    for t in ts:
        if t is not None and (not t.is_cuda or not t.is_contiguous()):
            raise ValueError("libmcg arguments must be contiguous CUDA tensors")


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def mcg_version() -> int:
    return _lib.mcg_version()


def mcg_release() -> None:
    _check("mcg_release", _lib.mcg_release())


def mcg_pack_links(canon: torch.Tensor, dims, precision=F64, stream=None) -> torch.Tensor:
    """canonical complex128 (nf, V, 4, 3, 3) -> SoA links."""
    _need_cuda(canon)
    assert canon.dtype == torch.complex128
    nf = canon.shape[0]
    U = empty_links(dims, nf, precision, canon.device)
    _check("mcg_pack_links", _lib.mcg_pack_links(_ptr(canon), _ptr(U), lattice(dims, nf, precision), _stream(stream)))
    return U


def mcg_unpack_links(U: torch.Tensor, dims, stream=None) -> torch.Tensor:
    _need_cuda(U)
    nf = U.shape[0]
    canon = torch.empty((nf, 2 * vh_of(dims), 4, 3, 3), dtype=torch.complex128, device=U.device)
    _check("mcg_unpack_links",
           _lib.mcg_unpack_links(_ptr(U), _ptr(canon), lattice(dims, nf, precision_of(U)), _stream(stream)))
    return canon


def mcg_pack_gauge(canon: torch.Tensor, dims, precision=F64, stream=None) -> torch.Tensor:
    _need_cuda(canon)
    assert canon.dtype == torch.complex128
    nf = canon.shape[0]
    G = empty_gauge(dims, nf, precision, canon.device)
    _check("mcg_pack_gauge", _lib.mcg_pack_gauge(_ptr(canon), _ptr(G), lattice(dims, nf, precision), _stream(stream)))
    return G


def mcg_unpack_gauge(G: torch.Tensor, dims, stream=None) -> torch.Tensor:
    _need_cuda(G)
    nf = G.shape[0]
    canon = torch.empty((nf, 2 * vh_of(dims), 3, 3), dtype=torch.complex128, device=G.device)
    _check("mcg_unpack_gauge",
           _lib.mcg_unpack_gauge(_ptr(G), _ptr(canon), lattice(dims, nf, precision_of(G)), _stream(stream)))
    return canon


def mcg_unpack_center(Z: torch.Tensor, dims, stream=None) -> torch.Tensor:
    _need_cuda(Z)
    nf = Z.shape[0]
    canon = torch.empty((nf, 2 * vh_of(dims), 4), dtype=torch.int8, device=Z.device)
    _check("mcg_unpack_center", _lib.mcg_unpack_center(_ptr(Z), _ptr(canon), lattice(dims, nf, F64), _stream(stream)))
    return canon


def mcg_convert(src: torch.Tensor, dst_precision: int, stream=None) -> torch.Tensor:
    _need_cuda(src)
    dst = torch.empty(src.shape, dtype=_real_dtype(dst_precision), device=src.device)
    _check("mcg_convert", _lib.mcg_convert(_ptr(src), precision_of(src), _ptr(dst), dst_precision,
                                           src.numel() // 2, _stream(stream)))
    return dst


def mcg_set_identity_gauge(G: torch.Tensor, dims, stream=None) -> torch.Tensor:
    _need_cuda(G)
    _check("mcg_set_identity_gauge",
           _lib.mcg_set_identity_gauge(_ptr(G), lattice(dims, G.shape[0], precision_of(G)), _stream(stream)))
    return G


def identity_gauge(dims, nfields=1, precision=F64, device="cuda") -> torch.Tensor:
    return mcg_set_identity_gauge(empty_gauge(dims, nfields, precision, device), dims)


def mcg_plaquette(U: torch.Tensor, dims, stream=None):
    _need_cuda(U)
    nf = U.shape[0]
    out = (ctypes.c_double * nf)()
    _check("mcg_plaquette", _lib.mcg_plaquette(_ptr(U), out, lattice(dims, nf, precision_of(U)), _stream(stream)))
    return list(out)


def mcg_functional(U: torch.Tensor, dims, stream=None):
    _need_cuda(U)
    nf = U.shape[0]
    out = (ctypes.c_double * nf)()
    _check("mcg_functional", _lib.mcg_functional(_ptr(U), out, lattice(dims, nf, precision_of(U)), _stream(stream)))
    return list(out)


def mcg_apply_gauge(U: torch.Tensor, G: torch.Tensor, dims, stream=None) -> torch.Tensor:
    _need_cuda(U, G)
    _check("mcg_apply_gauge",
           _lib.mcg_apply_gauge(_ptr(U), _ptr(G), lattice(dims, U.shape[0], precision_of(U)), _stream(stream)))
    return U


def mcg_reunitarise(M: torch.Tensor, which: int, dims, stream=None) -> torch.Tensor:
    _need_cuda(M)
    _check("mcg_reunitarise",
           _lib.mcg_reunitarise(_ptr(M), int(which), lattice(dims, M.shape[0], precision_of(M)), _stream(stream)))
    return M


def mcg_smear(U_in: torch.Tensor, dims, rho: float, eps: float, n: int, U_out: torch.Tensor | None = None,
              stream=None) -> torch.Tensor:
    _need_cuda(U_in)
    if U_out is None:
        U_out = torch.empty_like(U_in)
    _check("mcg_smear", _lib.mcg_smear(_ptr(U_in), _ptr(U_out), lattice(dims, U_in.shape[0], precision_of(U_in)),
                                       float(rho), float(eps), int(n), _stream(stream)))
    return U_out


def mcg_fix(U: torch.Tensor, G: torch.Tensor, dims, params: Params | None = None, history: bool = False,
            stream=None) -> dict:
    """MCG relaxation in place on U and G.  Returns dict(R, sweeps, converged, R_hist)."""
    _need_cuda(U, G)
    params = params or Params()
    nf = U.shape[0]
    R = (ctypes.c_double * nf)()
    sw = (ctypes.c_int * nf)()
    hist = (ctypes.c_double * (nf * (params.max_sweeps + 1)))() if history else None
    cp = params.c()
    rc = _check("mcg_fix", _lib.mcg_fix(_ptr(U), _ptr(G), lattice(dims, nf, precision_of(U)), ctypes.byref(cp), R, sw,
                                        hist, _stream(stream)), allow=(OK, NOT_CONVERGED))
    out = dict(R=list(R), sweeps=list(sw), converged=(rc == OK))
    if history:
        import numpy as np

        h = np.ctypeslib.as_array(hist).reshape(nf, params.max_sweeps + 1).copy()
        out["R_hist"] = [h[f, : sw[f] + 1] for f in range(nf)]
    return out


def mcg_center_project(U: torch.Tensor, dims, Z: torch.Tensor | None = None, stream=None):
    """Returns (Z, counts) with counts a list per field of [total, 01, 02, 03, 12, 13, 23]."""
    _need_cuda(U)
    nf = U.shape[0]
    if Z is None:
        Z = torch.empty((nf, 4, 2, vh_of(dims)), dtype=torch.int8, device=U.device)
    counts = (ctypes.c_longlong * (7 * nf))()
    _check("mcg_center_project",
           _lib.mcg_center_project(_ptr(U), _ptr(Z), counts, lattice(dims, nf, precision_of(U)), _stream(stream)))
    return Z, [list(counts[7 * f: 7 * f + 7]) for f in range(nf)]


def anneal_schedule(T0: float, T1: float, nsweeps: int) -> list:
    """Geometric temperatures from T0 (first sweep) to T1 (last sweep)."""
    if nsweeps < 1:
        return []
    if nsweeps == 1:
        return [float(T0)]
    r = (float(T1) / float(T0)) ** (1.0 / (nsweeps - 1))
    return [float(T0) * r**k for k in range(nsweeps)]


def mcg_anneal(U: torch.Tensor, G: torch.Tensor, dims, T, nhit: int = 4, eps: float = 0.3, seed: int = 0,
               first_sweep: int = 0, stream=None) -> dict:
    """Simulated annealing of the gauge transform in place on U and G (FP64),
    one sweep per temperature in T (see `anneal_schedule`); run mcg_fix
    afterwards to reach the nearest maximum.  Returns dict(accepted,
    acceptance) per field."""
    _need_cuda(U, G)
    nf = U.shape[0]
    Ts = (ctypes.c_double * max(1, len(T)))(*[float(t) for t in T])
    acc = (ctypes.c_longlong * nf)()
    _check("mcg_anneal", _lib.mcg_anneal(_ptr(U), _ptr(G), lattice(dims, nf, precision_of(U)), Ts, len(T),
                                         int(first_sweep), int(nhit), float(eps), int(seed) & ((1 << 64) - 1), acc,
                                         _stream(stream)))
    hits = len(T) * 3 * int(nhit) * 2 * vh_of(dims)
    return dict(accepted=list(acc), acceptance=[a / hits if hits else 0.0 for a in acc])


def mcg_random_gauge(dims, nfields: int = 1, seed: int = 0, seq: int = 0, device="cuda", stream=None) -> torch.Tensor:
    """Haar-random SU(3) gauge transforms (FP64 library layout), drawn on
    the device from Philox4x64-10 (see include/mcg.h); the same in each of the
    nfields fields."""
    G = empty_gauge(dims, nfields, F64, device)
    _check("mcg_random_gauge", _lib.mcg_random_gauge(_ptr(G), lattice(dims, nfields, F64),
                                                     int(seed) & ((1 << 64) - 1), int(seq) & ((1 << 64) - 1),
                                                     _stream(stream)))
    return G


def mcg_local_solve(A: torch.Tensor, b: torch.Tensor, precision: int = F64, stream=None):
    """Maximise a^T A a + 2 b.a over the unit sphere for a batch of local
    problems (the subgroup step of the relaxation, Sec. II.A) with the solve of
    the FP32 sweeps (precision F32) or of the exact FP64 sweep (F64).  A: (n, 4,
    4) float64 CUDA tensor (upper triangle read), b: (n, 4).  Returns (a (n, 4)
    float64, fallback (n,) int32: 1 where the Newton path gave way to Jacobi +
    secular)."""
    _need_cuda(A, b)
    if A.dtype != torch.float64 or b.dtype != torch.float64 or A.shape[1:] != (4, 4) or b.shape != (A.shape[0], 4):
        raise ValueError("A must be (n, 4, 4) and b (n, 4), float64")
    n = A.shape[0]
    a = torch.empty((n, 4), dtype=torch.float64, device=A.device)
    fb = torch.empty((n,), dtype=torch.int32, device=A.device)
    _check("mcg_local_solve", _lib.mcg_local_solve(_ptr(A), _ptr(b), _ptr(a), _ptr(fb), int(n), int(precision),
                                                   _stream(stream)))
    return a, fb


def mcg_vortex_remove(U: torch.Tensor, Z: torch.Tensor, dims, removed: bool = True, center: bool = True,
                      stream=None):
    """Center decomposition of a fixed field (Sec. III.A) with its center
    sectors Z: returns (U_removed = Z^dag U, U_center = Z * 1), each None when
    not requested."""
    _need_cuda(U, Z)
    if Z.dtype != torch.int8:
        raise TypeError("Z must be int8 center sectors")
    Ur = torch.empty_like(U) if removed else None
    Zl = torch.empty_like(U) if center else None
    _check("mcg_vortex_remove",
           _lib.mcg_vortex_remove(_ptr(U), _ptr(Z), _ptr(Ur) if Ur is not None else None,
                                  _ptr(Zl) if Zl is not None else None, lattice(dims, U.shape[0], precision_of(U)),
                                  _stream(stream)))
    return Ur, Zl


def mcg_wilson_loops(U: torch.Tensor, dims, Rmax: int, Tmax: int, stream=None):
    """Planar on-axis Wilson loops W(R, T) (Sec. III.A), averaged over all
    translations and the three spatial axes; numpy array (nfields, Rmax, Tmax)."""
    import numpy as np

    _need_cuda(U)
    nf = U.shape[0]
    out = (ctypes.c_double * (nf * Rmax * Tmax))()
    _check("mcg_wilson_loops", _lib.mcg_wilson_loops(_ptr(U), lattice(dims, nf, precision_of(U)), int(Rmax), int(Tmax),
                                                     out, _stream(stream)))
    return np.ctypeslib.as_array(out).reshape(nf, Rmax, Tmax).copy()


def mcg_wilson_loops_offaxis(U: torch.Tensor, dims, vectors, Tmax: int, stream=None):
    """Wilson loops with (possibly off-axis) spatial side r for each integer
    3-vector of `vectors`, averaged over translations and cubic images
    (Sec. III.A); numpy array (nfields, len(vectors), Tmax)."""
    import numpy as np

    _need_cuda(U)
    v = np.ascontiguousarray(np.asarray(vectors, dtype=np.int32).reshape(-1, 3))
    nf, nv = U.shape[0], v.shape[0]
    out = (ctypes.c_double * (nf * nv * Tmax))()
    _check("mcg_wilson_loops_offaxis",
           _lib.mcg_wilson_loops_offaxis(_ptr(U), lattice(dims, nf, precision_of(U)),
                                         v.ctypes.data_as(ctypes.c_void_p), nv, int(Tmax), out, _stream(stream)))
    return np.ctypeslib.as_array(out).reshape(nf, nv, Tmax).copy()


def mcg_precondition_fix(U: torch.Tensor, G: torch.Tensor, dims, params: Params | None = None, rho: float = 0.1,
                         eps: float = 1.0, nsmear: int = 0, smear_precision: int | None = None,
                         Z: torch.Tensor | None = None, stream=None) -> list:
    """Sec. II.B pipeline in place (U -> fixed field, G -> total transform)."""
    _need_cuda(U, G, Z)
    params = params or Params()
    nf = U.shape[0]
    prec = precision_of(U)
    res = (mcg_precond_result * nf)()
    cp = params.c()
    _check("mcg_precondition_fix",
           _lib.mcg_precondition_fix(_ptr(U), _ptr(G), _ptr(Z), lattice(dims, nf, prec), ctypes.byref(cp), float(rho),
                                     float(eps), int(nsmear), prec if smear_precision is None else int(smear_precision),
                                     res, _stream(stream)), allow=(OK, NOT_CONVERGED))
    return [r.as_dict() for r in res]


def mcg_precondition_levels(U: torch.Tensor, dims, nsmear, params: Params | None = None, rho: float = 0.1,
                            eps: float = 1.0, smear_precision: int | None = None, U_out: torch.Tensor | None = None,
                            G_out: torch.Tensor | None = None, Z_out: torch.Tensor | None = None,
                            stream=None):
    """Batched Sec. II.B scan over smearing levels of one field.
    Returns (U_out, G_out, Z_out, results)."""
    _need_cuda(U)
    params = params or Params()
    prec = precision_of(U)
    nl = len(nsmear)
    if U_out is None:
        U_out = empty_links(dims, nl, prec, U.device)
    if G_out is None:
        G_out = empty_gauge(dims, nl, prec, U.device)
    if Z_out is None:
        Z_out = torch.empty((nl, 4, 2, vh_of(dims)), dtype=torch.int8, device=U.device)
    _need_cuda(U_out, G_out, Z_out)
    ns = (ctypes.c_int * nl)(*[int(n) for n in nsmear])
    res = (mcg_precond_result * nl)()
    cp = params.c()
    _check("mcg_precondition_levels",
           _lib.mcg_precondition_levels(_ptr(U), _ptr(U_out), _ptr(G_out), _ptr(Z_out), lattice(dims, 1, prec),
                                        ctypes.byref(cp), float(rho), float(eps), ns, nl,
                                        prec if smear_precision is None else int(smear_precision), res,
                                        _stream(stream)), allow=(OK, NOT_CONVERGED))
    return U_out, G_out, Z_out, [r.as_dict() for r in res]


def mcg_time_halfsweep(U: torch.Tensor, G: torch.Tensor, dims, parity: int = 1, nreps: int = 10,
                       flush_l2: bool = True, stream=None) -> float:
    """Mean per-launch milliseconds of the half-sweep kernel (CUDA events)."""
    _need_cuda(U, G)
    ms = ctypes.c_float(0)
    _check("mcg_time_halfsweep", _lib.mcg_time_halfsweep(_ptr(U), _ptr(G), lattice(dims, 1, precision_of(U)),
                                                         int(parity), int(nreps), int(bool(flush_l2)),
                                                         ctypes.byref(ms), _stream(stream)))
    return ms.value


def mcg_halfsweep_slab(U: torch.Tensor, G: torch.Tensor, dims, parity: int, t_lo: int, t_hi: int,
                       want_R: bool = False, stream=None):
    """FP64 half-sweep of the sites of `parity` with t_lo <= t < t_hi (one
    field, in place); returns R over the updated sites' links if want_R."""
    _need_cuda(U, G)
    R = ctypes.c_double(0.0)
    _check("mcg_halfsweep_slab", _lib.mcg_halfsweep_slab(_ptr(U), _ptr(G), lattice(dims, 1, F64), int(parity),
                                                         int(t_lo), int(t_hi), ctypes.byref(R) if want_R else None,
                                                         _stream(stream)))
    return R.value if want_R else None


def mcg_slab_face(U: torch.Tensor, buf: torch.Tensor, dims, t: int, parity: int, to_field: bool,
                  precision: int = None, stream=None) -> torch.Tensor:
    """Copy the t-links of the parity-`parity` sites of layer t between the
    field U and the device buffer buf (9 * Nx*Ny*Nz/2 complex entries,
    entry-major, sites in (x, y, z) order); to_field=False reads the face
    into buf, True writes buf into U.  Returns buf."""
    _need_cuda(U, buf)
    prec = precision_of(U) if precision is None else precision
    n = dims[0] * dims[1] * dims[2] // 2
    need = 9 * n * (16 if prec == F64 else 8)
    if not buf.is_contiguous() or buf.numel() * buf.element_size() < need:
        raise ValueError(f"face buffer must be contiguous and hold {need} bytes")
    _check("mcg_slab_face", _lib.mcg_slab_face(_ptr(U), _ptr(buf), lattice(dims, 1, prec), int(t), int(parity),
                                               int(bool(to_field)), _stream(stream)))
    return buf


def mcg_bounds_violations(reset: bool = False) -> int:
    """Out-of-range indices the kernels met (index-checking build), -1 in a
    regular build."""
    return int(_lib.mcg_bounds_violations(int(bool(reset))))


def mcg_probe_peaks(stream=None) -> dict:
    """Measured FMA throughput of the device (TFLOP/s): FP64, FP32, packed FP32."""
    out = (ctypes.c_double * 3)()
    _check("mcg_probe_peaks", _lib.mcg_probe_peaks(out, _stream(stream)))
    return {"fp64_tflops": out[0], "fp32_tflops": out[1], "fp32x2_tflops": out[2]}


def mcg_kernel_launches() -> int:
    return int(_lib.mcg_kernel_launches())


def mcg_phase_stats(reset: bool = False) -> dict:
    """GPU milliseconds and site-updates of the FP64 and FP32 sweep phases
    since the last reset (CUDA events around the sweep graphs)."""
    ms = (ctypes.c_double * 2)()
    su = (ctypes.c_longlong * 2)()
    _check("mcg_phase_stats", _lib.mcg_phase_stats(ms, su, int(bool(reset))))
    return {"f64": {"ms": ms[0], "site_updates": su[0]}, "f32": {"ms": ms[1], "site_updates": su[1]}}


def mcg_plaquette_static(U: torch.Tensor, dims, out: torch.Tensor, stream=None) -> torch.Tensor:
    """Mean plaquette per field into the caller's float64 CUDA tensor `out`
    (nfields entries); the library allocates nothing for this call (its
    partial sums live in a fixed array inside libmcg).  Asynchronous."""
    _need_cuda(U, out)
    if out.dtype != torch.float64 or out.numel() < U.shape[0]:
        raise ValueError("out must be a float64 CUDA tensor with one entry per field")
    _check("mcg_plaquette_static",
           _lib.mcg_plaquette_static(_ptr(U), _ptr(out), lattice(dims, U.shape[0], precision_of(U)), _stream(stream)))
    return out


def mcg_set_sweep_block(precision: int, threads: int) -> None:
    _check("mcg_set_sweep_block", _lib.mcg_set_sweep_block(int(precision), int(threads)))


def mcg_get_sweep_block(precision: int) -> int:
    return int(_lib.mcg_get_sweep_block(int(precision)))


def autotune_sweep_block(U: torch.Tensor, dims, reps: int = 10) -> dict:
    """Pick the half-sweep block size for U's precision (64/128 threads for
    FP64, 64/128/256 for FP32; one thread per site) by timing each on a
    scratch copy of U (L2 flushed between launches); keeps the fastest for the
    process and returns the timings in ms per launch."""
    prec = precision_of(U)
    Uc = U[:1].clone()
    G = identity_gauge(dims, 1, prec, U.device)
    times = {}
    for nt in ((64, 128, 256) if prec == F32 else (64, 128)):
        mcg_set_sweep_block(prec, nt)
        mcg_time_halfsweep(Uc, G, dims, 1, 2, True)  # warm-up
        times[nt] = 0.5 * (mcg_time_halfsweep(Uc, G, dims, 1, reps, True) +
                           mcg_time_halfsweep(Uc, G, dims, 0, reps, True))
    best = min(times, key=times.get)
    mcg_set_sweep_block(prec, best)
    return {"chosen": best, "ms_per_launch": times}


def _field_array(Us, Gs, dims_list):
    n = len(Us)
    arr = (mcg_field * n)()
    for k, (U, G, d) in enumerate(zip(Us, Gs, dims_list)):
        _need_cuda(U, G)
        arr[k].U = U.data_ptr()
        arr[k].G = G.data_ptr()
        for j in range(4):
            arr[k].dims[j] = int(d[j])
    return arr


def mcg_fix_batch(Us, Gs, dims_list, params: Params | None = None, stream=None) -> dict:
    """MCG relaxation of fields of any sizes in one batch (in place).  Us, Gs:
    single-field tensors (1, ...) of one precision.  Returns dict(R, sweeps, converged)."""
    params = params or Params()
    n = len(Us)
    prec = precision_of(Us[0])
    arr = _field_array(Us, Gs, dims_list)
    R = (ctypes.c_double * n)()
    sw = (ctypes.c_int * n)()
    cp = params.c()
    rc = _check("mcg_fix_batch", _lib.mcg_fix_batch(arr, n, prec, ctypes.byref(cp), R, sw, _stream(stream)),
                allow=(OK, NOT_CONVERGED))
    return dict(R=list(R), sweeps=list(sw), converged=(rc == OK))


def mcg_gribov_search(Us, Gs, dims_list, config_of_copy, nconfigs: int, params: Params | None = None,
                      stream=None) -> dict:
    """Gribov-copy search in place: U_k (the configuration's links) and G_k (a
    random initial transform) per copy; returns dict(R, sweeps, best_copy,
    best_V, converged) with best_copy[c] the copy of configuration c with the
    largest V_U."""
    params = params or Params()
    n = len(Us)
    prec = precision_of(Us[0])
    arr = _field_array(Us, Gs, dims_list)
    cfg = (ctypes.c_int * n)(*[int(c) for c in config_of_copy])
    R = (ctypes.c_double * n)()
    sw = (ctypes.c_int * n)()
    best = (ctypes.c_int * nconfigs)()
    bestV = (ctypes.c_double * nconfigs)()
    cp = params.c()
    rc = _check("mcg_gribov_search",
                _lib.mcg_gribov_search(arr, n, cfg, int(nconfigs), prec, ctypes.byref(cp), R, sw, best, bestV,
                                       _stream(stream)), allow=(OK, NOT_CONVERGED))
    return dict(R=list(R), sweeps=list(sw), best_copy=list(best), best_V=list(bestV), converged=(rc == OK))


def autotune_schedule(Us, dims_list, params: Params, trial_sweeps: int = 40,
                      chunks=(10, 25, 50)) -> dict:
    """Tile and sweep-schedule autotuner for a batch: for every half-sweep
    block size of the sweep precision and every graph chunk length
    (check_every), time `trial_sweeps` sweeps of mcg_fix_batch on clones of
    the batch (no stop test), keep the fastest: the block size is set for the
    process, the chunk length is returned in params.check_every.  Only the
    clones are modified."""
    prec = F32 if (params.fp32_sweeps > 0 or precision_of(Us[0]) == F32) else F64
    Uc = [mcg_convert(U, F32) if prec == F32 and precision_of(U) == F64 else U.clone() for U in Us]
    Gc = [identity_gauge(d, 1, prec, U.device) for U, d in zip(Uc, dims_list)]
    blocks = (64, 128, 256) if prec == F32 else (64, 128)
    best = None
    timings = {}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for nt in blocks:
        mcg_set_sweep_block(prec, nt)
        for ch in chunks:
            p = Params(tol=-1e300, max_sweeps=trial_sweeps, check_every=ch, reunit_every=params.reunit_every)
            mcg_fix_batch(Uc, Gc, dims_list, p)  # warm-up: graph build, caches
            ev0.record()
            mcg_fix_batch(Uc, Gc, dims_list, p)
            ev1.record()
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1) / trial_sweeps
            timings[f"{nt}x{ch}"] = ms
            if best is None or ms < best[0]:
                best = (ms, nt, ch)
    mcg_set_sweep_block(prec, best[1])
    params.check_every = best[2]
    return {"precision": "f32" if prec == F32 else "f64", "block": best[1], "check_every": best[2],
            "ms_per_sweep": timings}


# ---------------------------------------------------------------------------
# differentiation
# ---------------------------------------------------------------------------
def mcg_smear_backward_step(U: torch.Tensor, Gout: torch.Tensor, dims, rho: float, eps: float,
                            stream=None) -> torch.Tensor:
    """Gradient w.r.t. the input U of one smearing step, given the gradient
    Gout w.r.t. its output (FP64, link layout)."""
    _need_cuda(U, Gout)
    if U.dtype != torch.float64 or Gout.dtype != torch.float64:
        raise TypeError("the smearing backward runs on FP64 fields and gradients")
    Gin = torch.empty_like(Gout)
    _check("mcg_smear_backward_step",
           _lib.mcg_smear_backward_step(_ptr(U), _ptr(Gout), _ptr(Gin), lattice(dims, U.shape[0], F64), float(rho),
                                        float(eps), _stream(stream)))
    return Gin


def mcg_functional_matrix_grad(U: torch.Tensor, dims, stream=None) -> torch.Tensor:
    _need_cuda(U)
    G = torch.empty(U.shape, dtype=torch.float64, device=U.device)
    _check("mcg_functional_matrix_grad",
           _lib.mcg_functional_matrix_grad(_ptr(U), _ptr(G), lattice(dims, U.shape[0], precision_of(U)),
                                           _stream(stream)))
    return G


def mcg_grad_R(U: torch.Tensor, dims, stream=None) -> torch.Tensor:
    """dR/d eps_a(x) for Omega(x) -> exp(i eps lambda_a/2) Omega(x): (nfields, V, 8) FP64."""
    _need_cuda(U)
    nf = U.shape[0]
    grad = torch.empty((nf, 2 * vh_of(dims), 8), dtype=torch.float64, device=U.device)
    _check("mcg_grad_R", _lib.mcg_grad_R(_ptr(U), _ptr(grad), lattice(dims, nf, precision_of(U)), _stream(stream)))
    return grad


def mcg_ascent_step(U: torch.Tensor, G: torch.Tensor, grad: torch.Tensor, dims, alpha: float, stream=None):
    _need_cuda(U, G, grad)
    _check("mcg_ascent_step", _lib.mcg_ascent_step(_ptr(U), _ptr(G), _ptr(grad), float(alpha),
                                                   lattice(dims, U.shape[0], precision_of(U)), _stream(stream)))
    return U, G


class StoutSmear(torch.autograd.Function):
    """U -> smear(U, rho, eps, n) with the hand-written backward: the n
    intermediate fields are kept (full checkpointing) and the steps are
    differentiated in reverse by mcg_smear_backward_step.  FP64 only."""

    @staticmethod
    def forward(ctx, U, dims, rho, eps, n):
        fields = [U]
        for _ in range(int(n)):
            fields.append(mcg_smear(fields[-1], dims, rho, eps, 1))
        ctx.save_for_backward(*fields[:-1])
        ctx.params = (tuple(dims), float(rho), float(eps))
        return fields[-1] if n > 0 else U.clone()

    @staticmethod
    def backward(ctx, grad_out):
        dims, rho, eps = ctx.params
        G = grad_out.contiguous().to(torch.float64)
        for Uk in reversed(ctx.saved_tensors):
            G = mcg_smear_backward_step(Uk, G, dims, rho, eps)
        return G, None, None, None, None


class MCGFunctional(torch.autograd.Function):
    """R(U) = sum |tr U_mu(x)|^2 per field with its matrix-gradient backward."""

    @staticmethod
    def forward(ctx, U, dims):
        ctx.save_for_backward(U)
        ctx.dims = tuple(dims)
        return torch.tensor(mcg_functional(U, dims), dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(ctx, gR):
        (U,) = ctx.saved_tensors
        G = mcg_functional_matrix_grad(U, ctx.dims)
        return G * gR.view(-1, *([1] * (G.dim() - 1))), None


def ascent_refine(U: torch.Tensor, G: torch.Tensor, dims, steps: int = 20, alpha: float = 0.05,
                  min_alpha: float = 1e-8) -> dict:
    """Gradient-ascent refinement of the MCG functional over the gauge
    transform (in place on U, G): each step moves along dR/d eps with step
    alpha, halving alpha whenever R would fall (the trial runs on clones)."""
    R = mcg_functional(U, dims)[0]
    hist = [R]
    for _ in range(int(steps)):
        grad = mcg_grad_R(U, dims)
        while alpha >= min_alpha:
            Ut, Gt = U.clone(), G.clone()
            mcg_ascent_step(Ut, Gt, grad, dims, alpha)
            Rt = mcg_functional(Ut, dims)[0]
            if Rt >= R:
                U.copy_(Ut)
                G.copy_(Gt)
                R = Rt
                hist.append(R)
                alpha *= 1.5
                break
            alpha *= 0.5
        else:
            break
    return {"R": R, "R_hist": hist, "alpha": alpha}
