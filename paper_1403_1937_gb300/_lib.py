"""ctypes binding of libeik.so (the C ABI declared in include/eik.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
If the shared object is missing, loading fails loudly; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libeik.so")

EIK_OK = 0
EIK_ERR_ARG = 1
EIK_ERR_CUDA = 2
EIK_ERR_OOM = 3
EIK_ERR_NOT_CONVERGED = 4
EIK_ERR_BREAKDOWN = 5
EIK_ERR_TIMEOUT = 6
EIK_ERR_STATE = 7

STATUS_NAMES = {
    0: "EIK_OK", 1: "EIK_ERR_ARG", 2: "EIK_ERR_CUDA", 3: "EIK_ERR_OOM",
    4: "EIK_ERR_NOT_CONVERGED", 5: "EIK_ERR_BREAKDOWN", 6: "EIK_ERR_TIMEOUT",
    7: "EIK_ERR_STATE",
}

PREC_FP64 = 0
PREC_MIXED = 1
STOP_COMPONENTWISE = 0
STOP_NORMWISE = 1
PRECOND_JACOBI = 0
PRECOND_MULTIGRID = 1
BOUNDARY_HALF_CELL = 0
BOUNDARY_DROP_EDGE = 1


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tol", ctypes.c_double),
                ("stop_norm", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("boundary", ctypes.c_int), ("tile_override", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("band_bits", ctypes.c_int), ("test_flags", ctypes.c_int),
                ("batch_pack", ctypes.c_int), ("batch_tile_rows", ctypes.c_int),
                ("precond", ctypes.c_int), ("reserved", ctypes.c_int * 2)]


class Stats(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int),
                ("res_cw", ctypes.c_double), ("res_nw", ctypes.c_double),
                ("ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64),
                ("timed_launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class EikError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

# (name, restype, argtypes) of every exported entry point
_P = ctypes.c_void_p
_SIGS = [
    ("eik_default_options", None, [ctypes.POINTER(Options)]),
    ("eik_create", ctypes.c_int,
     [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_double,
      ctypes.c_double, _P, _P, _P, ctypes.c_int64, ctypes.POINTER(Options), _P]),
    ("eik_set_f", ctypes.c_int, [_P, _P]),
    ("eik_solve", ctypes.c_int, [_P, _P, _P, ctypes.POINTER(Stats)]),
    ("eik_grad", ctypes.c_int, [_P, _P, _P, ctypes.POINTER(Stats)]),
    ("eik_destroy", ctypes.c_int, [_P]),
    ("eik_set_profiling", ctypes.c_int, [_P, ctypes.c_int]),
    ("eik_kernel_stats", ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("eik_reset_kernel_stats", ctypes.c_int, [_P]),
    ("eik_create_batch", ctypes.c_int,
     [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _P, _P, _P, _P,
      ctypes.POINTER(Options), _P]),
    ("eik_set_f_batch", ctypes.c_int, [_P, _P]),
    ("eik_solve_batch", ctypes.c_int, [_P, _P, _P]),
    ("eik_grad_batch", ctypes.c_int, [_P, _P, _P, _P]),
    ("eik_destroy_batch", ctypes.c_int, [_P]),
    ("eik_batch_set_concurrency", ctypes.c_int, [_P, ctypes.c_int]),
    ("eik_batch_info", ctypes.c_int,
     [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
      ctypes.POINTER(ctypes.c_double)]),
    ("eik_residual_noalloc", ctypes.c_int,
     [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_double, ctypes.c_double, _P, _P,
      _P, ctypes.c_int64, ctypes.c_int, _P, _P]),
    ("eik_grad_S", ctypes.c_int,
     [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_double, _P, _P, _P]),
    ("eik_backtrack", ctypes.c_int,
     [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_double, _P, _P, ctypes.c_int64,
      ctypes.c_double, ctypes.c_int, _P, ctypes.c_int64, ctypes.c_double, _P, _P, _P, _P]),
    ("eik_sfs_forcing", ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double, _P, _P]),
    ("eik_fft_series", ctypes.c_int,
     [ctypes.POINTER(ctypes.c_int64), ctypes.c_double, ctypes.c_double, _P, _P, ctypes.c_int64,
      ctypes.c_int, ctypes.c_double, _P, _P, ctypes.POINTER(ctypes.c_double), _P]),
    ("eik_last_error", ctypes.c_char_p, []),
    ("eik_abi_version", ctypes.c_int, []),
    ("eik_cuda_arch", ctypes.c_int, []),
]


def lib_path() -> str:
    return LIB_PATH


def load():
    """Loads libeik.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is missing: build it with `python -m "
            "paper_1403_1937_gb300.build` (or __graft_entry__.build())")
    lib = ctypes.CDLL(LIB_PATH)
    for name, res, args in _SIGS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def last_error() -> str:
    return load().eik_last_error().decode()


def check(status: int, allow=(EIK_OK,)):
    if status not in allow:
        raise EikError(status, last_error())
    return status


def default_options() -> Options:
    o = Options()
    load().eik_default_options(ctypes.byref(o))
    return o
