"""CPU oracle for the Jacobi-preconditioned CG solve (test infrastructure).

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline may import this package; the product path never does.  The
arithmetic lives in ``oracle.c`` (plain sequential C, FP64 unless a
function says otherwise); this module compiles it with gcc and marshals
numpy arrays through ctypes.  It shares no code with the CUDA library.

Citations (paper sections): MatMult on MATAIJ (Sec. 4), VecAXPY/VecDot/
VecNorm (Sec. 5.1 and the Sec. 2 stub routine), PCJACOBI (Sec. 5.3), KSPCG
(Sec. 5.5), single precision on the GPU with FP64 elsewhere (Response A7,
Sec. 4).  The CG iteration itself is the textbook one (Saad, Algorithm 9.1)
because the paper does not print it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CONVERGED = 0
DIVERGED_ITS = 1
ERR_ARG = -1
ERR_DIAG = -4
ERR_INDEFINITE = -5
ERR_NAN = -6
ERR_STAGNATION = -8
ERR_CSR = -10

# -O2 without fast-math and without FMA contraction keeps every operation a
# correctly rounded IEEE operation in the written order, on x86 and Arm alike.
CFLAGS = ["-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fno-fast-math"]


def _compile(out: str, extra, force: bool) -> str:
    with _lock:
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
            tmp = out + f".{os.getpid()}.tmp"
            subprocess.run(["gcc", *CFLAGS, *extra, _SRC, "-o", tmp, "-lm"], check=True)
            os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc)."""
    return _compile(_LIB, [], force)


_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lib_omp = None


def build_omp(force: bool = False) -> str:
    """The same source built with OpenMP (liboracle_omp.so): its SpMV and
    vector loops run on all host cores.  Used only to time the oracle on
    every core (the CPU baseline); nothing is checked against it."""
    return _compile(_LIB_OMP, ["-fopenmp"], force)


def pcg_threaded(A, b, rtol, maxit):
    """oracle pcg() through the OpenMP build, for timing on all host cores.
    Returns dict(status, iters, rnorm, threads)."""
    global _lib_omp
    if _lib_omp is None:
        build_omp()
        lib = ctypes.CDLL(_LIB_OMP)
        i64, vp = ctypes.c_int64, ctypes.c_void_p
        lib.orc_pcg.argtypes = [i64, vp, vp, vp, vp, vp, ctypes.c_double, i64,
                                ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double), vp]
        lib.orc_pcg.restype = ctypes.c_int
        lib.orc_threads.restype = ctypes.c_int
        _lib_omp = lib
    rp, ci, v, bb = _i32(A.rowptr), _i32(A.colidx), _f64(A.vals), _f64(b)
    x = np.zeros(A.n)
    it = ctypes.c_int64(0)
    rn = ctypes.c_double(0.0)
    st = _lib_omp.orc_pcg(A.n, _p(rp), _p(ci), _p(v), _p(bb), _p(x), float(rtol), int(maxit),
                          ctypes.byref(it), ctypes.byref(rn), None)
    threads = int(_lib_omp.orc_threads())
    return {"status": st, "iters": it.value, "rnorm": rn.value, "threads": threads}


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, i32p, f64p = ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p
        lib.orc_csr_check.argtypes = [i64, i64, i32p, i32p]
        lib.orc_csr_check.restype = ctypes.c_int
        lib.orc_spmv.argtypes = [i64, i32p, i32p, f64p, f64p, f64p]
        lib.orc_spmv_f32.argtypes = [i64, i32p, i32p, f64p, f64p, f64p]
        lib.orc_dot.argtypes = [i64, f64p, f64p]
        lib.orc_dot.restype = ctypes.c_double
        lib.orc_dot2.argtypes = [i64, f64p, f64p]
        lib.orc_dot2.restype = ctypes.c_double
        lib.orc_norm2.argtypes = [i64, f64p]
        lib.orc_norm2.restype = ctypes.c_double
        lib.orc_axpy.argtypes = [i64, ctypes.c_double, f64p, f64p]
        lib.orc_aypx.argtypes = [i64, ctypes.c_double, f64p, f64p]
        lib.orc_axpy_fused.argtypes = [i64, ctypes.c_double, f64p, f64p]
        lib.orc_aypx_fused.argtypes = [i64, ctypes.c_double, f64p, f64p]
        lib.orc_jacobi_dinv.argtypes = [i64, i32p, i32p, f64p, f64p]
        lib.orc_jacobi_dinv.restype = ctypes.c_int
        lib.orc_pcg.argtypes = [i64, i32p, i32p, f64p, f64p, f64p, ctypes.c_double, i64,
                                ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double), f64p]
        lib.orc_pcg.restype = ctypes.c_int
        lib.orc_pcg_norm.argtypes = [i64, i32p, i32p, f64p, f64p, f64p, ctypes.c_double, i64,
                                     ctypes.c_int, ctypes.POINTER(i64),
                                     ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double), f64p]
        lib.orc_pcg_norm.restype = ctypes.c_int
        lib.orc_chebyshev.argtypes = [i64, i32p, i32p, f64p, f64p, f64p, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, i64,
                                      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                                      f64p]
        lib.orc_chebyshev.restype = ctypes.c_int
        lib.orc_coo_to_csr.argtypes = [i64, i64, i64, i32p, i32p, f64p, i32p, i32p, f64p,
                                       ctypes.POINTER(ctypes.c_int64)]
        lib.orc_coo_to_csr.restype = ctypes.c_int
        lib.orc_pcg_f32.argtypes = [i64, i32p, i32p, f64p, f64p, f64p, f64p, ctypes.c_float, i64,
                                    ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_float)]
        lib.orc_pcg_f32.restype = ctypes.c_int
        lib.orc_pcg_mixed.argtypes = [i64, i32p, i32p, f64p, f64p, f64p, ctypes.c_double,
                                      ctypes.c_double, i64, i64, ctypes.POINTER(i64),
                                      ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double)]
        lib.orc_pcg_mixed.restype = ctypes.c_int
        lib.orc_block_pcg.argtypes = [i64, i32p, i32p, f64p, ctypes.c_int, f64p, f64p,
                                      ctypes.c_double, i64, ctypes.POINTER(i64), f64p, f64p]
        lib.orc_block_pcg.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def csr_check(n, ncols, rowptr, colidx) -> int:
    rp, ci = _i32(rowptr), _i32(colidx)
    return _load().orc_csr_check(n, ncols, _p(rp), _p(ci))


def spmv(A, x) -> np.ndarray:
    """y = A x in FP64 (A: object with n, rowptr, colidx, vals)."""
    rp, ci, v, xx = _i32(A.rowptr), _i32(A.colidx), _f64(A.vals), _f64(x)
    y = np.empty(A.n)
    _load().orc_spmv(A.n, _p(rp), _p(ci), _p(v), _p(xx), _p(y))
    return y


def spmv_f32(A, x) -> np.ndarray:
    """y = A x with FP32 values, vector and accumulation."""
    rp, ci, v, xx = _i32(A.rowptr), _i32(A.colidx), _f32(A.vals), _f32(x)
    y = np.empty(A.n, dtype=np.float32)
    _load().orc_spmv_f32(A.n, _p(rp), _p(ci), _p(v), _p(xx), _p(y))
    return y


def dot(x, y) -> float:
    xx, yy = _f64(x), _f64(y)
    return _load().orc_dot(len(xx), _p(xx), _p(yy))


def dot2(x, y) -> float:
    xx, yy = _f64(x), _f64(y)
    return _load().orc_dot2(len(xx), _p(xx), _p(yy))


def norm2(x) -> float:
    xx = _f64(x)
    return _load().orc_norm2(len(xx), _p(xx))


def axpy(alpha, x, y) -> np.ndarray:
    """Returns alpha x + y (y is copied, not modified)."""
    xx, yy = _f64(x), _f64(y).copy()
    _load().orc_axpy(len(xx), alpha, _p(xx), _p(yy))
    return yy


def aypx(beta, x, y) -> np.ndarray:
    """Returns x + beta y (y is copied, not modified)."""
    xx, yy = _f64(x), _f64(y).copy()
    _load().orc_aypx(len(xx), beta, _p(xx), _p(yy))
    return yy


def axpy_fused(alpha, x, y) -> np.ndarray:
    """Returns alpha x + y with one rounding per entry (fused multiply-add)."""
    xx, yy = _f64(x), _f64(y).copy()
    _load().orc_axpy_fused(len(xx), alpha, _p(xx), _p(yy))
    return yy


def aypx_fused(beta, x, y) -> np.ndarray:
    """Returns x + beta y with one rounding per entry (fused multiply-add)."""
    xx, yy = _f64(x), _f64(y).copy()
    _load().orc_aypx_fused(len(xx), beta, _p(xx), _p(yy))
    return yy


def jacobi_dinv(A):
    """(status, dinv) with dinv_i = 1/a_ii."""
    rp, ci, v = _i32(A.rowptr), _i32(A.colidx), _f64(A.vals)
    d = np.zeros(A.n)
    st = _load().orc_jacobi_dinv(A.n, _p(rp), _p(ci), _p(v), _p(d))
    return st, d


def pcg(A, b, rtol, maxit, x0=None, history=False, norm=0):
    """Jacobi-PCG in FP64 with the stopping test N(r) <= rtol N(b) in norm
    0 (||v||_2), 1 (||D^-1 v||_2) or 2 (sqrt(v . D^-1 v)).  Returns
    dict(x, status, iters, rnorm, bnorm[, rhist])."""
    rp, ci, v, bb = _i32(A.rowptr), _i32(A.colidx), _f64(A.vals), _f64(b)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    it = ctypes.c_int64(0)
    rn = ctypes.c_double(0.0)
    bn = ctypes.c_double(0.0)
    rh = np.full(maxit + 1, np.nan) if history else None
    st = _load().orc_pcg_norm(A.n, _p(rp), _p(ci), _p(v), _p(bb), _p(x), float(rtol), int(maxit),
                              int(norm), ctypes.byref(it), ctypes.byref(rn), ctypes.byref(bn),
                              _p(rh) if history else None)
    out = {"x": x, "status": st, "iters": it.value, "rnorm": rn.value, "bnorm": bn.value}
    if history:
        out["rhist"] = rh[: it.value + 1]
    return out


def chebyshev(A, b, emin, emax, rtol, maxit, x0=None, history=False):
    """Jacobi-preconditioned Chebyshev iteration for a spectrum of D^-1 A in
    [emin, emax], in FP64.  Returns dict(x, status, iters, rnorm[, rhist])."""
    rp, ci, v, bb = _i32(A.rowptr), _i32(A.colidx), _f64(A.vals), _f64(b)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    it = ctypes.c_int64(0)
    rn = ctypes.c_double(0.0)
    rh = np.full(maxit + 1, np.nan) if history else None
    st = _load().orc_chebyshev(A.n, _p(rp), _p(ci), _p(v), _p(bb), _p(x), float(emin), float(emax),
                               float(rtol), int(maxit), ctypes.byref(it), ctypes.byref(rn),
                               _p(rh) if history else None)
    out = {"x": x, "status": st, "iters": it.value, "rnorm": rn.value}
    if history:
        out["rhist"] = rh[: it.value + 1]
    return out


def coo_to_csr(nrows, ncols, ti, tj, v):
    """Returns (status, rowptr, colidx, vals): triplets (ti, tj, v) assembled
    into CSR, duplicates summed in triplet order."""
    ti, tj, v = _i32(ti), _i32(tj), _f64(v)
    m = len(ti)
    rowptr = np.zeros(nrows + 1, dtype=np.int32)
    colidx = np.zeros(max(m, 1), dtype=np.int32)
    vals = np.zeros(max(m, 1))
    nout = ctypes.c_int64(0)
    st = _load().orc_coo_to_csr(int(nrows), int(ncols), m, _p(ti), _p(tj), _p(v), _p(rowptr),
                                _p(colidx), _p(vals), ctypes.byref(nout))
    return st, rowptr, colidx[: nout.value].copy(), vals[: nout.value].copy()


def pcg_f32(A, b, rtol, maxit):
    """Jacobi-PCG entirely in FP32 from x0 = 0."""
    st0, dinv = jacobi_dinv(A)
    if st0:
        return {"status": st0, "iters": 0, "rnorm": 0.0, "x": np.zeros(A.n, np.float32)}
    rp, ci = _i32(A.rowptr), _i32(A.colidx)
    v32, d32, bb = _f32(A.vals), _f32(dinv), _f32(b)
    x = np.zeros(A.n, dtype=np.float32)
    it = ctypes.c_int64(0)
    rn = ctypes.c_float(0.0)
    st = _load().orc_pcg_f32(A.n, _p(rp), _p(ci), _p(v32), _p(d32), _p(bb), _p(x),
                             float(rtol), int(maxit), ctypes.byref(it), ctypes.byref(rn))
    return {"x": x, "status": st, "iters": it.value, "rnorm": rn.value}


def pcg_mixed(A, b, rtol, inner_rtol=1e-4, inner_maxit=10000, outer_maxit=30, x0=None):
    """FP32-inner PCG with FP64 iterative refinement."""
    rp, ci, v, bb = _i32(A.rowptr), _i32(A.colidx), _f64(A.vals), _f64(b)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    o = ctypes.c_int64(0)
    i = ctypes.c_int64(0)
    rn = ctypes.c_double(0.0)
    st = _load().orc_pcg_mixed(A.n, _p(rp), _p(ci), _p(v), _p(bb), _p(x), float(rtol),
                               float(inner_rtol), int(inner_maxit), int(outer_maxit),
                               ctypes.byref(o), ctypes.byref(i), ctypes.byref(rn))
    return {"x": x, "status": st, "outer": o.value, "inner": i.value, "rnorm": rn.value}


def block_pcg(A, B, rtol, maxit, X0=None):
    """Block Jacobi-PCG (O'Leary) in FP64 for the k columns of B (an n x k
    array, or k * n values column by column).  Returns dict(x (n x k),
    status, iters (block iterations), rnorm[k], bnorm[k])."""
    rp, ci, v = _i32(A.rowptr), _i32(A.colidx), _f64(A.vals)
    Bc = np.asfortranarray(np.asarray(B, dtype=np.float64).reshape(A.n, -1, order="F"))
    k = Bc.shape[1]
    bb = np.ascontiguousarray(Bc.T).reshape(-1)          # column j at j * n
    X = np.zeros(A.n * k) if X0 is None else np.ascontiguousarray(
        np.asarray(X0, dtype=np.float64).reshape(A.n, -1, order="F").T).reshape(-1).copy()
    it = ctypes.c_int64(0)
    rn = np.zeros(k)
    bn = np.zeros(k)
    st = _load().orc_block_pcg(A.n, _p(rp), _p(ci), _p(v), int(k), _p(bb), _p(X), float(rtol),
                               int(maxit), ctypes.byref(it), _p(rn), _p(bn))
    return {"x": X.reshape(k, A.n).T.copy(), "status": st, "iters": it.value, "rnorm": rn,
            "bnorm": bn}
