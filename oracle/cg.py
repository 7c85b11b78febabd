"""ctypes front end of the C oracle CG (``oracle/cg.c``).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  The shared object is
built in-tree under ``oracle/_build`` with gcc and OpenMP, on demand or by
``__graft_entry__.build()``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

from . import fd

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cg.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle_cg.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle/cg.c into oracle/_build/liboracle_cg.so."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC",
                           "-std=c11", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_pcg.restype = ctypes.c_int
        lib.oracle_pcg.argtypes = [ctypes.c_int64, i64p, i64p, dp, dp, dp,
                                   ctypes.c_double, ctypes.c_int64,
                                   ctypes.c_int64, ctypes.c_int, i64p, dp]
        lib.oracle_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def threads() -> int:
    return int(_load().oracle_threads())


def pcg(A, b, x0=None, tol=1e-13, max_iter=100000, min_iter=0, nthreads=0):
    """Jacobi-PCG on a scipy sparse matrix.  Returns (x, status, iters, cw)."""
    lib = _load()
    A = A.tocsr()
    A.sort_indices()
    n = A.shape[0]
    ip = np.ascontiguousarray(A.indptr, dtype=np.int64)
    ix = np.ascontiguousarray(A.indices, dtype=np.int64)
    v = np.ascontiguousarray(A.data, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = (np.zeros(n) if x0 is None
         else np.ascontiguousarray(x0, dtype=np.float64).copy())
    it = ctypes.c_int64(0)
    cw = ctypes.c_double(0.0)
    i64p = ctypes.POINTER(ctypes.c_int64)
    dp = ctypes.POINTER(ctypes.c_double)
    st = lib.oracle_pcg(n, ip.ctypes.data_as(i64p), ix.ctypes.data_as(i64p),
                        v.ctypes.data_as(dp), b.ctypes.data_as(dp),
                        x.ctypes.data_as(dp), float(tol), int(max_iter),
                        int(min_iter), int(nthreads), ctypes.byref(it),
                        ctypes.byref(cw))
    return x, int(st), int(it.value), float(cw.value)


def solve(f, dims, h, hbar, src_idx, src_U=None, boundary=0, tol=1e-13,
          max_iter=200000, min_iter=0, nthreads=0):
    """Full solve through the CG oracle.  Returns (S, phi_shifted, system,
    info) with info = dict(status, iters, cw)."""
    sys = fd.assemble(f, dims, h, hbar, src_idx, src_U, boundary)
    x, st, it, cw = pcg(sys.A, sys.b, tol=tol, max_iter=max_iter,
                        min_iter=min_iter, nthreads=nthreads)
    phi = fd.full_phi(sys, x)
    return fd.S_from_phi(sys, phi), phi, sys, dict(status=st, iters=it, cw=cw)


def time_iterations(sys, iters: int, nthreads: int = 0):
    """Run exactly ``iters`` CG iterations (tolerance 0) from x = 0 and return
    the wall time in seconds; used for the CPU baseline throughput."""
    t0 = time.perf_counter()
    pcg(sys.A, sys.b, tol=0.0, max_iter=iters, min_iter=iters,
        nthreads=nthreads)
    return time.perf_counter() - t0
