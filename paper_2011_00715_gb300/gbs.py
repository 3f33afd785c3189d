"""Python binding of the gbs C ABI (include/gbs.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Arrays are
numpy arrays (host memory) or torch tensors (host or CUDA); their memory
space is stated to the library explicitly, never queried.  Negative status
codes raise :class:`GbsError`, except from the solve calls, which return
their status inside the result because breakdown and limit statuses are
results, not misuse.

The library must have been built (``paper_2011_00715_gb300.build.build()``
or ``__graft_entry__.build()``); there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

GBS_OK = 0
GBS_DIVERGED_ITS = 1
GBS_ERR_ARG = -1
GBS_ERR_OOM = -2
GBS_ERR_CUDA = -3
GBS_ERR_DIAG = -4
GBS_ERR_INDEFINITE = -5
GBS_ERR_NAN = -6
GBS_ERR_TIMEOUT = -7
GBS_ERR_STAGNATION = -8
GBS_ERR_BUDGET = -9
GBS_ERR_CSR = -10
GBS_ERR_NOT_FOUND = -11
GBS_ERR_UNSUPPORTED = -12

GBS_MEM_HOST = 0
GBS_MEM_DEVICE = 1
GBS_F64 = 0
GBS_F32 = 1
GBS_MODE_FP64 = 0
GBS_MODE_MIXED = 1
GBS_ALG_AUTO = 0
GBS_ALG_PERSISTENT = 1
GBS_ALG_PEROP = 2
GBS_ALG_GRAPH = 3
GBS_ALG_CLUSTER = 4
GBS_NORM_UNPRECONDITIONED = 0
GBS_NORM_PRECONDITIONED = 1
GBS_NORM_NATURAL = 2
GBS_CLUSTER_MAX_ROWS = 32768
GBS_NOALLOC_MAX_ROWS = 262144


class GbsError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {gbs_status_string(status)} ({status})")


class gbs_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("algorithm", ctypes.c_int),
                ("inner_rtol", ctypes.c_double), ("outer_maxit", ctypes.c_int),
                ("barrier_timeout_ms", ctypes.c_int), ("graph_iters", ctypes.c_int),
                ("fault_skip_arrival", ctypes.c_int), ("batched_lanes", ctypes.c_int),
                ("persistent_ctas", ctypes.c_int), ("norm_type", ctypes.c_int),
                ("no_rel16", ctypes.c_int), ("persistent_shape", ctypes.c_int),
                ("persistent_lanes", ctypes.c_int), ("spmv_lanes", ctypes.c_int),
                ("reserved", ctypes.c_int * 1)]


class gbs_solve_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("rnorm", ctypes.c_double), ("bnorm", ctypes.c_double),
                ("device_ms", ctypes.c_double), ("model_bytes", ctypes.c_double),
                ("cta_threads", ctypes.c_int), ("lanes_per_row", ctypes.c_int)]


@dataclass
class SolveInfo:
    status: int
    iters: int
    outer_iters: int
    rnorm: float
    bnorm: float
    device_ms: float
    model_bytes: float = 0.0
    cta_threads: int = 0
    lanes_per_row: int = 0


_lib = None
_VP = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32P = ctypes.POINTER(ctypes.c_int)

_SIGS = {
    "gbs_version": ([], ctypes.c_char_p),
    "gbs_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "gbs_opts_default": ([ctypes.POINTER(gbs_opts)], ctypes.c_int),
    "gbs_ctx_create": ([ctypes.c_int, _VP, ctypes.POINTER(gbs_opts), ctypes.POINTER(_VP)], ctypes.c_int),
    "gbs_ctx_destroy": ([_VP], ctypes.c_int),
    "gbs_ctx_set_stream": ([_VP, _VP], ctypes.c_int),
    "gbs_ctx_set_opts": ([_VP, ctypes.POINTER(gbs_opts)], ctypes.c_int),
    "gbs_ctx_synchronize": ([_VP], ctypes.c_int),
    "gbs_ctx_launch_count": ([_VP, ctypes.POINTER(_I64)], ctypes.c_int),
    "gbs_probe_fp64_rate": ([_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "gbs_mat_create_aij": ([_VP, _I64, _I64, _VP, _VP, _VP, ctypes.c_int, ctypes.POINTER(_VP)], ctypes.c_int),
    "gbs_mat_set_values": ([_VP, _VP, ctypes.c_int], ctypes.c_int),
    "gbs_mat_create_coo": ([_VP, _I64, _I64, _I64, _VP, _VP, _VP, ctypes.c_int, ctypes.POINTER(_VP)],
                           ctypes.c_int),
    "gbs_mat_set_values_coo": ([_VP, _VP, ctypes.c_int], ctypes.c_int),
    "gbs_mat_get_csr": ([_VP, _VP, _VP, _VP, ctypes.c_int], ctypes.c_int),
    "gbs_mat_get_info": ([_VP, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64)], ctypes.c_int),
    "gbs_mat_get_device": ([_VP, _I32P], ctypes.c_int),
    "gbs_mat_destroy": ([_VP], ctypes.c_int),
    "gbs_mat_mult": ([_VP, _VP, _VP], ctypes.c_int),
    "gbs_vec_create": ([_VP, _I64, ctypes.c_int, ctypes.POINTER(_VP)], ctypes.c_int),
    "gbs_vec_wrap": ([_VP, _VP, _I64, ctypes.c_int, ctypes.POINTER(_VP)], ctypes.c_int),
    "gbs_vec_destroy": ([_VP], ctypes.c_int),
    "gbs_vec_get_info": ([_VP, ctypes.POINTER(_I64), _I32P, ctypes.POINTER(_VP)], ctypes.c_int),
    "gbs_vec_set_values": ([_VP, _VP, ctypes.c_int], ctypes.c_int),
    "gbs_vec_get_values": ([_VP, _VP, ctypes.c_int], ctypes.c_int),
    "gbs_vec_set": ([_VP, ctypes.c_double], ctypes.c_int),
    "gbs_vec_copy": ([_VP, _VP], ctypes.c_int),
    "gbs_vec_axpy": ([_VP, ctypes.c_double, _VP], ctypes.c_int),
    "gbs_vec_aypx": ([_VP, ctypes.c_double, _VP], ctypes.c_int),
    "gbs_vec_pointwise_mult": ([_VP, _VP, _VP], ctypes.c_int),
    "gbs_vec_dot": ([_VP, _VP, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "gbs_vec_norm2": ([_VP, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "gbs_vec_dot_async": ([_VP, _VP, _VP], ctypes.c_int),
    "gbs_vec_norm2_async": ([_VP, _VP], ctypes.c_int),
    "gbs_pc_jacobi_create": ([_VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "gbs_pc_apply": ([_VP, _VP, _VP], ctypes.c_int),
    "gbs_pc_destroy": ([_VP], ctypes.c_int),
    "gbs_ksp_solve_cg": ([_VP, _VP, _VP, ctypes.c_double, ctypes.c_int, _I32P,
                          ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "gbs_ksp_solve_cg_ex": ([_VP, _VP, _VP, ctypes.c_double, ctypes.c_int, ctypes.POINTER(gbs_opts),
                             ctypes.POINTER(gbs_solve_info)], ctypes.c_int),
    "gbs_ksp_last_info": ([_VP, ctypes.POINTER(gbs_solve_info)], ctypes.c_int),
    "gbs_ksp_solve_chebyshev": ([_VP, _VP, _VP, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int, ctypes.POINTER(gbs_solve_info)], ctypes.c_int),
    "gbs_ksp_solve_cg_noalloc": ([_VP, _VP, _VP, ctypes.c_double, ctypes.c_int,
                                  ctypes.POINTER(gbs_solve_info)], ctypes.c_int),
    "gbs_ksp_solve_cg_batched": ([_VP, ctypes.c_int, _VP, _VP, _VP, _VP, _VP, ctypes.c_int,
                                  ctypes.c_int, _VP, _VP, _VP], ctypes.c_int),
    "gbs_server_create": ([_VP, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_VP)], ctypes.c_int),
    "gbs_server_destroy": ([_VP], ctypes.c_int),
    "gbs_server_submit": ([_VP, _I64, _VP, _VP, _VP, ctypes.c_int, _VP, ctypes.c_double, ctypes.c_int,
                           ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "gbs_server_submit_borrowed": ([_VP, _I64, _VP, _VP, _VP, ctypes.c_int, _VP, ctypes.c_double,
                                    ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "gbs_batched_tune": ([_VP, _VP, ctypes.c_int, ctypes.c_int, _I32P], ctypes.c_int),
    "gbs_ksp_tune": ([_VP, ctypes.c_int, _I32P, _I32P], ctypes.c_int),
    "gbs_ksp_solve_cg_block": ([_VP, ctypes.c_int, _VP, _VP, ctypes.c_double, ctypes.c_int,
                                ctypes.POINTER(gbs_solve_info), _VP], ctypes.c_int),
    "gbs_server_progress": ([_VP, _I32P], ctypes.c_int),
    "gbs_server_poll": ([_VP, ctypes.c_uint64, _I32P], ctypes.c_int),
    "gbs_server_wait": ([_VP, ctypes.c_uint64], ctypes.c_int),
    "gbs_server_fetch": ([_VP, ctypes.c_uint64, _VP, _VP, _VP, _VP], ctypes.c_int),
    "gbs_server_stats": ([_VP, _I32P, _I32P, _I32P, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "gbs_server_times": ([_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
}


def library_path() -> str:
    return _build.OUT


def lib():
    """The loaded libgbs.so.  Raises if it has not been built: there is no
    CPU fallback for any operation."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise ImportError(f"libgbs.so is not built ({path}); run "
                              "paper_2011_00715_gb300.build.build()")
        L = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(st: int, where: str) -> int:
    if st < 0:
        raise GbsError(st, where)
    return st


def _ptr_space(a):
    """(pointer, memspace, keepalive) of a numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return a.ctypes.data, GBS_MEM_HOST, a
    import torch
    if isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), (GBS_MEM_DEVICE if a.is_cuda else GBS_MEM_HOST), a
    raise TypeError(f"unsupported array type {type(a)}")


def _dtype_code(a) -> int:
    s = str(a.dtype)
    if s.endswith("float64"):
        return GBS_F64
    if s.endswith("float32"):
        return GBS_F32
    raise TypeError(f"unsupported dtype {a.dtype}")


# ---------------------------------------------------------------- general --

def gbs_version() -> str:
    return lib().gbs_version().decode()


def gbs_status_string(status: int) -> str:
    return lib().gbs_status_string(int(status)).decode()


def gbs_opts_default(**overrides) -> gbs_opts:
    o = gbs_opts()
    _check(lib().gbs_opts_default(ctypes.byref(o)), "gbs_opts_default")
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


# -------------------------------------------------------------------- ctx --

def gbs_ctx_create(device: int = 0, stream=None, opts: gbs_opts | None = None):
    """stream: a cudaStream_t as int (e.g. torch.cuda.current_stream().cuda_stream)."""
    h = _VP()
    _check(lib().gbs_ctx_create(device, _VP(stream or 0), ctypes.byref(opts) if opts else None,
                                ctypes.byref(h)), "gbs_ctx_create")
    return h


def gbs_ctx_destroy(ctx):
    _check(lib().gbs_ctx_destroy(ctx), "gbs_ctx_destroy")


def gbs_ctx_set_stream(ctx, stream):
    _check(lib().gbs_ctx_set_stream(ctx, _VP(stream or 0)), "gbs_ctx_set_stream")


def gbs_ctx_set_opts(ctx, opts: gbs_opts):
    _check(lib().gbs_ctx_set_opts(ctx, ctypes.byref(opts)), "gbs_ctx_set_opts")


def gbs_ctx_synchronize(ctx):
    _check(lib().gbs_ctx_synchronize(ctx), "gbs_ctx_synchronize")


def gbs_probe_fp64_rate(ctx, iters: int = 4096) -> float:
    """FP64 FMAs per second of the device (a timed FMA-chain kernel)."""
    r = ctypes.c_double()
    _check(lib().gbs_probe_fp64_rate(ctx, iters, ctypes.byref(r)), "gbs_probe_fp64_rate")
    return r.value


def gbs_ctx_launch_count(ctx) -> int:
    c = _I64()
    _check(lib().gbs_ctx_launch_count(ctx, ctypes.byref(c)), "gbs_ctx_launch_count")
    return c.value


# ----------------------------------------------------------------- matrix --

def gbs_mat_create_aij(ctx, nrows: int, ncols: int, rowptr, colidx, vals):
    """rowptr/colidx int32, vals float64: all numpy/host or all CUDA tensors."""
    p_rp, s_rp, _k1 = _ptr_space(rowptr)
    p_ci, s_ci, _k2 = _ptr_space(colidx)
    p_v, s_v, _k3 = _ptr_space(vals)
    if not (s_rp == s_ci == s_v):
        raise ValueError("rowptr, colidx and vals must live in the same memory space")
    if str(rowptr.dtype).split(".")[-1] != "int32" or str(colidx.dtype).split(".")[-1] != "int32":
        raise TypeError("rowptr and colidx must be int32")
    if _dtype_code(vals) != GBS_F64:
        raise TypeError("vals must be float64")
    h = _VP()
    _check(lib().gbs_mat_create_aij(ctx, nrows, ncols, _VP(p_rp), _VP(p_ci), _VP(p_v), s_rp,
                                    ctypes.byref(h)), "gbs_mat_create_aij")
    return h


def gbs_mat_set_values(A, vals):
    p, s, _k = _ptr_space(vals)
    _check(lib().gbs_mat_set_values(A, _VP(p), s), "gbs_mat_set_values")


def gbs_mat_create_coo(ctx, nrows: int, ncols: int, i, j, v):
    """Device assembly from triplets (i, j int32, v float64; all numpy/host
    or all CUDA tensors); repeated (row, column) pairs summed in order."""
    p_i, s_i, _k1 = _ptr_space(i)
    p_j, s_j, _k2 = _ptr_space(j)
    p_v, s_v, _k3 = _ptr_space(v)
    if not (s_i == s_j == s_v):
        raise ValueError("i, j and v must live in the same memory space")
    if str(i.dtype).split(".")[-1] != "int32" or str(j.dtype).split(".")[-1] != "int32":
        raise TypeError("i and j must be int32")
    if _dtype_code(v) != GBS_F64:
        raise TypeError("v must be float64")
    if not (len(i) == len(j) == len(v)):
        raise ValueError("i, j and v must have the same length")
    h = _VP()
    _check(lib().gbs_mat_create_coo(ctx, int(nrows), int(ncols), len(i), _VP(p_i), _VP(p_j), _VP(p_v),
                                    s_i, ctypes.byref(h)), "gbs_mat_create_coo")
    return h


def gbs_mat_set_values_coo(A, v):
    p, s, _k = _ptr_space(v)
    _check(lib().gbs_mat_set_values_coo(A, _VP(p), s), "gbs_mat_set_values_coo")


def gbs_mat_get_csr(A):
    """(rowptr, colidx, vals) as host numpy arrays."""
    n, _m, nnz = gbs_mat_get_info(A)
    rp = np.empty(n + 1, dtype=np.int32)
    ci = np.empty(max(nnz, 1), dtype=np.int32)
    v = np.empty(max(nnz, 1))
    _check(lib().gbs_mat_get_csr(A, rp.ctypes.data, ci.ctypes.data, v.ctypes.data, GBS_MEM_HOST),
           "gbs_mat_get_csr")
    return rp, ci[:nnz], v[:nnz]


def gbs_mat_get_info(A):
    n, m, z = _I64(), _I64(), _I64()
    _check(lib().gbs_mat_get_info(A, ctypes.byref(n), ctypes.byref(m), ctypes.byref(z)),
           "gbs_mat_get_info")
    return n.value, m.value, z.value


def gbs_mat_get_device(A) -> int:
    d = ctypes.c_int32()
    _check(lib().gbs_mat_get_device(A, ctypes.byref(d)), "gbs_mat_get_device")
    return d.value


def gbs_mat_destroy(A):
    _check(lib().gbs_mat_destroy(A), "gbs_mat_destroy")


def gbs_mat_mult(A, x, y):
    _check(lib().gbs_mat_mult(A, x, y), "gbs_mat_mult")


# ----------------------------------------------------------------- vector --

def gbs_vec_create(ctx, n: int, dtype: int = GBS_F64):
    h = _VP()
    _check(lib().gbs_vec_create(ctx, n, dtype, ctypes.byref(h)), "gbs_vec_create")
    return h


def gbs_vec_wrap(ctx, tensor):
    """Wrap a contiguous CUDA tensor (float64 or float32) without copying; the
    caller keeps the tensor alive while the handle is used."""
    p, s, _k = _ptr_space(tensor)
    if s != GBS_MEM_DEVICE:
        raise ValueError("gbs_vec_wrap needs device memory")
    h = _VP()
    _check(lib().gbs_vec_wrap(ctx, _VP(p), tensor.numel(), _dtype_code(tensor), ctypes.byref(h)),
           "gbs_vec_wrap")
    return h


def gbs_vec_destroy(v):
    _check(lib().gbs_vec_destroy(v), "gbs_vec_destroy")


def gbs_vec_get_info(v):
    n, d, p = _I64(), ctypes.c_int(), _VP()
    _check(lib().gbs_vec_get_info(v, ctypes.byref(n), ctypes.byref(d), ctypes.byref(p)),
           "gbs_vec_get_info")
    return n.value, d.value, p.value


def gbs_vec_set_values(v, src):
    p, s, _k = _ptr_space(src)
    _check(lib().gbs_vec_set_values(v, _VP(p), s), "gbs_vec_set_values")


def gbs_vec_get_values(v, dst):
    p, s, _k = _ptr_space(dst)
    _check(lib().gbs_vec_get_values(v, _VP(p), s), "gbs_vec_get_values")
    return dst


def gbs_vec_set(v, alpha: float):
    _check(lib().gbs_vec_set(v, float(alpha)), "gbs_vec_set")


def gbs_vec_copy(x, y):
    _check(lib().gbs_vec_copy(x, y), "gbs_vec_copy")


def gbs_vec_axpy(y, alpha: float, x):
    _check(lib().gbs_vec_axpy(y, float(alpha), x), "gbs_vec_axpy")


def gbs_vec_aypx(y, beta: float, x):
    _check(lib().gbs_vec_aypx(y, float(beta), x), "gbs_vec_aypx")


def gbs_vec_pointwise_mult(w, x, y):
    _check(lib().gbs_vec_pointwise_mult(w, x, y), "gbs_vec_pointwise_mult")


def gbs_vec_dot(x, y) -> float:
    out = ctypes.c_double()
    _check(lib().gbs_vec_dot(x, y, ctypes.byref(out)), "gbs_vec_dot")
    return out.value


def gbs_vec_norm2(x) -> float:
    out = ctypes.c_double()
    _check(lib().gbs_vec_norm2(x, ctypes.byref(out)), "gbs_vec_norm2")
    return out.value


def _dev_scalar(out):
    """Device address of a CUDA float64 tensor with at least one element."""
    if getattr(out, "is_cuda", False) is not True or str(out.dtype) != "torch.float64" \
            or out.numel() < 1:
        raise ValueError("out must be a CUDA float64 tensor with at least one element")
    return _VP(out.data_ptr())


def gbs_vec_dot_async(x, y, out) -> None:
    """x . y written to out[0] (a CUDA float64 tensor) in stream order."""
    _check(lib().gbs_vec_dot_async(x, y, _dev_scalar(out)), "gbs_vec_dot_async")


def gbs_vec_norm2_async(x, out) -> None:
    """||x||_2 written to out[0] (a CUDA float64 tensor) in stream order."""
    _check(lib().gbs_vec_norm2_async(x, _dev_scalar(out)), "gbs_vec_norm2_async")


# --------------------------------------------------------- preconditioner --

def gbs_pc_jacobi_create(A):
    h = _VP()
    _check(lib().gbs_pc_jacobi_create(A, ctypes.byref(h)), "gbs_pc_jacobi_create")
    return h


def gbs_pc_apply(pc, r, z):
    _check(lib().gbs_pc_apply(pc, r, z), "gbs_pc_apply")


def gbs_pc_destroy(pc):
    _check(lib().gbs_pc_destroy(pc), "gbs_pc_destroy")


# ----------------------------------------------------------------- solver --

def _info(i: gbs_solve_info) -> SolveInfo:
    return SolveInfo(i.status, i.iters, i.outer_iters, i.rnorm, i.bnorm, i.device_ms, i.model_bytes,
                     i.cta_threads, i.lanes_per_row)


_RESULT_STATUSES = (GBS_OK, GBS_DIVERGED_ITS, GBS_ERR_DIAG, GBS_ERR_INDEFINITE, GBS_ERR_NAN,
                    GBS_ERR_TIMEOUT, GBS_ERR_STAGNATION)


def gbs_ksp_solve_cg(A, b, x, rtol: float, maxit: int):
    """Returns (status, iters, rnorm)."""
    it = ctypes.c_int()
    rn = ctypes.c_double()
    st = lib().gbs_ksp_solve_cg(A, b, x, float(rtol), int(maxit), ctypes.byref(it), ctypes.byref(rn))
    if st not in _RESULT_STATUSES:
        _check(st, "gbs_ksp_solve_cg")
    return st, it.value, rn.value


def gbs_ksp_solve_cg_ex(A, b, x, rtol: float, maxit: int, opts: gbs_opts | None = None) -> SolveInfo:
    info = gbs_solve_info()
    st = lib().gbs_ksp_solve_cg_ex(A, b, x, float(rtol), int(maxit),
                                   ctypes.byref(opts) if opts else None, ctypes.byref(info))
    if st not in _RESULT_STATUSES:
        _check(st, "gbs_ksp_solve_cg_ex")
    return _info(info)


def gbs_ksp_solve_chebyshev(A, b, x, emin: float, emax: float, rtol: float, maxit: int) -> SolveInfo:
    """Jacobi-preconditioned Chebyshev iteration for a spectrum of D^-1 A in
    [emin, emax].  Result statuses are returned in the SolveInfo."""
    info = gbs_solve_info()
    st = lib().gbs_ksp_solve_chebyshev(A, b, x, float(emin), float(emax), float(rtol), int(maxit),
                                       ctypes.byref(info))
    if st not in _RESULT_STATUSES:
        _check(st, "gbs_ksp_solve_chebyshev")
    return _info(info)


def gbs_ksp_solve_cg_block(A, k: int, B, X, rtol: float, maxit: int):
    """Block Jacobi-PCG for the k columns of B (a gbs_vec of n * k entries,
    column-major) into X.  Returns (SolveInfo, per-column final residual
    norms as a numpy array)."""
    info = gbs_solve_info()
    rn = np.zeros(int(k))
    st = lib().gbs_ksp_solve_cg_block(A, int(k), B, X, float(rtol), int(maxit), ctypes.byref(info),
                                      rn.ctypes.data)
    if st not in _RESULT_STATUSES:
        _check(st, "gbs_ksp_solve_cg_block")
    return _info(info), rn


def gbs_ksp_tune(A, mode: int):
    """(shape, lanes per row) the tuner picks for A's class in this mode."""
    sh, ln = ctypes.c_int(), ctypes.c_int()
    _check(lib().gbs_ksp_tune(A, int(mode), ctypes.byref(sh), ctypes.byref(ln)), "gbs_ksp_tune")
    return sh.value, ln.value


def gbs_ksp_last_info(ctx) -> SolveInfo:
    info = gbs_solve_info()
    _check(lib().gbs_ksp_last_info(ctx, ctypes.byref(info)), "gbs_ksp_last_info")
    return _info(info)


def gbs_ksp_solve_cg_noalloc(A, b, x, rtol: float, maxit: int) -> SolveInfo:
    """Allocation-free FP64 solve: b and x are caller-owned CUDA float64
    tensors of the matrix's size (see include/gbs.h for the limits)."""
    pb, sb, _kb = _ptr_space(b)
    px, sx, _kx = _ptr_space(x)
    if sb != GBS_MEM_DEVICE or sx != GBS_MEM_DEVICE:
        raise ValueError("b and x must be device tensors")
    if _dtype_code(b) != GBS_F64 or _dtype_code(x) != GBS_F64:
        raise TypeError("b and x must be float64")
    # the C entry point gets bare pointers: the length and the device are
    # checked here, where the tensors are known
    n, _m, _z = gbs_mat_get_info(A)
    if b.numel() != n or x.numel() != n:
        raise ValueError(f"b and x must have {n} entries (got {b.numel()} and {x.numel()})")
    dev = gbs_mat_get_device(A)
    if b.device.index != dev or x.device.index != dev:
        raise ValueError(f"b and x must be on cuda:{dev}, the matrix's device")
    info = gbs_solve_info()
    st = lib().gbs_ksp_solve_cg_noalloc(A, _VP(pb), _VP(px), float(rtol), int(maxit),
                                        ctypes.byref(info))
    if st not in _RESULT_STATUSES:
        _check(st, "gbs_ksp_solve_cg_noalloc")
    return _info(info)


def gbs_ksp_solve_cg_batched(ctx, mats, Bs, Xs, nrhs, rtols, maxit: int, mode: int):
    """Returns (status, iters[], rnorm[], status[]) per (system, column)."""
    ns = len(mats)
    A = (_VP * ns)(*mats)
    B = (_VP * ns)(*Bs)
    X = (_VP * ns)(*Xs)
    K = (ctypes.c_int * ns)(*[int(k) for k in nrhs])
    R = (ctypes.c_double * ns)(*[float(r) for r in rtols])
    tot = int(sum(int(k) for k in nrhs))
    its = np.zeros(tot, dtype=np.int32)
    rns = np.zeros(tot, dtype=np.float64)
    sts = np.zeros(tot, dtype=np.int32)
    st = lib().gbs_ksp_solve_cg_batched(ctx, ns, A, B, X, K, R, int(maxit), int(mode),
                                        its.ctypes.data, rns.ctypes.data, sts.ctypes.data)
    if st not in _RESULT_STATUSES:
        _check(st, "gbs_ksp_solve_cg_batched")
    return st, its, rns, sts


# ---------------------------------------------------------------- serving --

def gbs_batched_tune(ctx, A, k: int, mode: int = GBS_MODE_MIXED) -> int:
    """Lanes per row the batched engines use for systems like A (tuned once
    per class and context)."""
    lanes = ctypes.c_int()
    _check(lib().gbs_batched_tune(ctx, A, int(k), int(mode), ctypes.byref(lanes)),
           "gbs_batched_tune")
    return lanes.value


def gbs_server_create(ctx, hbm_budget_bytes: int, max_slots: int = 0, mode: int = GBS_MODE_MIXED):
    h = _VP()
    _check(lib().gbs_server_create(ctx, int(hbm_budget_bytes), int(max_slots), int(mode),
                                   ctypes.byref(h)), "gbs_server_create")
    return h


def gbs_server_destroy(srv):
    _check(lib().gbs_server_destroy(srv), "gbs_server_destroy")


def gbs_server_submit(srv, nrows: int, rowptr, colidx, vals, k: int, b, rtol: float, maxit: int) -> int:
    for a in (rowptr, colidx, vals, b):
        if not isinstance(a, np.ndarray) or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("server inputs are contiguous host numpy arrays")
    t = ctypes.c_uint64()
    _check(lib().gbs_server_submit(srv, int(nrows), rowptr.ctypes.data, colidx.ctypes.data,
                                   vals.ctypes.data, int(k), b.ctypes.data, float(rtol), int(maxit),
                                   ctypes.byref(t)), "gbs_server_submit")
    return t.value


def gbs_server_submit_borrowed(srv, nrows: int, rowptr, colidx, vals, k: int, b, rtol: float,
                               maxit: int) -> int:
    """As gbs_server_submit without the copy: the caller keeps the four
    arrays alive and unchanged until the request is done."""
    for a in (rowptr, colidx, vals, b):
        if not isinstance(a, np.ndarray) or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("server inputs are contiguous host numpy arrays")
    t = ctypes.c_uint64()
    _check(lib().gbs_server_submit_borrowed(srv, int(nrows), rowptr.ctypes.data, colidx.ctypes.data,
                                            vals.ctypes.data, int(k), b.ctypes.data, float(rtol),
                                            int(maxit), ctypes.byref(t)), "gbs_server_submit_borrowed")
    return t.value


def gbs_server_progress(srv) -> int:
    r = ctypes.c_int()
    _check(lib().gbs_server_progress(srv, ctypes.byref(r)), "gbs_server_progress")
    return r.value


def gbs_server_poll(srv, ticket: int) -> bool:
    d = ctypes.c_int()
    _check(lib().gbs_server_poll(srv, ctypes.c_uint64(ticket), ctypes.byref(d)), "gbs_server_poll")
    return bool(d.value)


def gbs_server_wait(srv, ticket: int):
    _check(lib().gbs_server_wait(srv, ctypes.c_uint64(ticket)), "gbs_server_wait")


def gbs_server_fetch(srv, ticket: int, n: int, k: int):
    """Returns (x[n*k], iters[k], rnorm[k], status[k])."""
    x = np.empty(n * k)
    its = np.zeros(k, dtype=np.int32)
    rns = np.zeros(k)
    sts = np.zeros(k, dtype=np.int32)
    _check(lib().gbs_server_fetch(srv, ctypes.c_uint64(ticket), x.ctypes.data, its.ctypes.data,
                                  rns.ctypes.data, sts.ctypes.data), "gbs_server_fetch")
    return x, its, rns, sts


def gbs_server_stats(srv):
    q, r, f = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    b = ctypes.c_size_t()
    _check(lib().gbs_server_stats(srv, ctypes.byref(q), ctypes.byref(r), ctypes.byref(f),
                                  ctypes.byref(b)), "gbs_server_stats")
    return q.value, r.value, f.value, b.value


def gbs_server_times(srv):
    """(admit_s, quanta_s, retire_s, quanta) since the server was created."""
    a, q, r = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    n = ctypes.c_int64()
    _check(lib().gbs_server_times(srv, ctypes.byref(a), ctypes.byref(q), ctypes.byref(r),
                                  ctypes.byref(n)), "gbs_server_times")
    return a.value, q.value, r.value, n.value
