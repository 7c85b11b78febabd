"""The C-ABI library builds, loads and exports every entry point that
include/eik.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "eik.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    names = set(re.findall(r"\b(eik_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1403_1937_gb300 import build
    build.build()
    from paper_1403_1937_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("eik_create", "eik_solve", "eik_grad", "eik_destroy", "eik_set_f",
                     "eik_last_error", "eik_default_options"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_binding_covers_the_header():
    from paper_1403_1937_gb300 import _lib
    bound = {name for name, _, _ in _lib._SIGS}
    assert set(declared_functions()) <= bound


def test_default_options_and_version(lib):
    from paper_1403_1937_gb300 import _lib
    o = _lib.default_options()
    assert o.precision == _lib.PREC_FP64
    assert o.tol == 1e-12
    assert o.stop_norm == _lib.STOP_COMPONENTWISE
    assert o.max_iter == 200000
    assert o.boundary == _lib.BOUNDARY_HALF_CELL
    assert lib.eik_abi_version() == 1
    assert lib.eik_cuda_arch() == 1030


def test_struct_layout_matches_header(tmp_path):
    """The ctypes mirrors of eik_options / eik_stats have the C compiler's
    sizes and field offsets."""
    import subprocess
    from paper_1403_1937_gb300 import _lib
    src = tmp_path / "layout.c"
    fields_o = [f for f, _ in _lib.Options._fields_]
    fields_s = [f for f, _ in _lib.Stats._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"',
             'int main(void) {',
             'printf("%zu\\n", sizeof(eik_options));',
             'printf("%zu\\n", sizeof(eik_stats));']
    lines += [f'printf("%zu\\n", offsetof(eik_options, {f}));' for f in fields_o]
    lines += [f'printf("%zu\\n", offsetof(eik_stats, {f}));' for f in fields_s]
    lines += ['return 0; }']
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", str(src), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(_lib.Options), ctypes.sizeof(_lib.Stats)]
    want += [getattr(_lib.Options, f).offset for f in fields_o]
    want += [getattr(_lib.Stats, f).offset for f in fields_s]
    assert vals == want


def test_null_arguments_rejected_without_gpu(lib):
    from paper_1403_1937_gb300 import _lib
    out = ctypes.c_void_p()
    st = lib.eik_create(ctypes.byref(out), 4, None, 1.0, 1.0, None, None, None, 1, None, None)
    assert st == _lib.EIK_ERR_ARG
    assert "ndim" in _lib.last_error()
    assert lib.eik_destroy(None) == _lib.EIK_OK


def test_preconditioner_option_checked_without_gpu(lib):
    """An unknown precond and multigrid in FP64 are rejected before any CUDA
    call."""
    from paper_1403_1937_gb300 import _lib
    P = ctypes.c_void_p(0x1000)      # never dereferenced: the checks fail first
    for ndim, prec, pc in ((2, _lib.PREC_MIXED, 2), (2, _lib.PREC_MIXED, -1),
                           (2, _lib.PREC_FP64, _lib.PRECOND_MULTIGRID),
                           (3, _lib.PREC_FP64, _lib.PRECOND_MULTIGRID)):
        o = _lib.default_options()
        o.precision = prec
        o.precond = pc
        dims = (ctypes.c_int64 * ndim)(*([9] * ndim))
        out = ctypes.c_void_p()
        st = lib.eik_create(ctypes.byref(out), ndim, dims, 0.1, 0.1, P, P, None, 1,
                            ctypes.byref(o), None)
        assert st == _lib.EIK_ERR_ARG, (ndim, prec, pc)
        assert "precond" in _lib.last_error() or "multigrid" in _lib.last_error()


def test_path_and_forcing_entry_points_validate_arguments_without_gpu(lib):
    """Argument checks of the path-planning, forcing and allocation-free
    entry points run before any CUDA call."""
    from paper_1403_1937_gb300 import _lib
    d1 = (ctypes.c_int64 * 1)(63)
    d2 = (ctypes.c_int64 * 2)(9, 7)
    dbad = (ctypes.c_int64 * 2)(1, 7)
    P = ctypes.c_void_p(0x1000)      # never dereferenced: the checks fail first
    assert lib.eik_grad_S(1, d1, 0.1, P, P, None) == _lib.EIK_ERR_ARG       # ndim
    assert lib.eik_grad_S(2, dbad, 0.1, P, P, None) == _lib.EIK_ERR_ARG     # size < 2
    assert lib.eik_grad_S(2, d2, 0.0, P, P, None) == _lib.EIK_ERR_ARG       # h <= 0
    assert lib.eik_grad_S(2, d2, 0.1, None, P, None) == _lib.EIK_ERR_ARG    # null S
    # step <= 0, eps < 0, max_steps < 0, npaths < 0
    for step, eps, ms, npaths in ((0.0, 0.1, 5, 1), (0.1, -1.0, 5, 1), (0.1, 0.1, -1, 1),
                                  (0.1, 0.1, 5, -1)):
        assert lib.eik_backtrack(2, d2, 0.1, P, P, npaths, step, ms, P, 1, eps, P, P, P,
                                 None) == _lib.EIK_ERR_ARG
    assert lib.eik_backtrack(2, d2, 0.1, P, P, 0, 0.1, 5, P, 1, 0.1, P, P, P,
                             None) == _lib.EIK_OK                           # nothing to do
    assert lib.eik_sfs_forcing(P, -1, 0.0, P, None) == _lib.EIK_ERR_ARG
    assert lib.eik_sfs_forcing(P, 4, -0.1, P, None) == _lib.EIK_ERR_ARG
    assert lib.eik_sfs_forcing(None, 4, 0.0, P, None) == _lib.EIK_ERR_ARG
    assert lib.eik_sfs_forcing(None, 0, 0.0, None, None) == _lib.EIK_OK
    big = (ctypes.c_int64 * 2)(1025, 1024)                                  # > 2^20 nodes
    res = ctypes.c_void_p(0x1000)
    assert lib.eik_residual_noalloc(2, big, 0.1, 0.1, P, P, P, 1, 0, res, None) == \
        _lib.EIK_ERR_ARG
    # extents whose product wraps around int64 to a small number (3 * 6148914691236517206
    # = 2 mod 2^64) are rejected before they are multiplied
    wrap = (ctypes.c_int64 * 2)(3, 6148914691236517206)
    assert lib.eik_residual_noalloc(2, wrap, 0.1, 0.1, P, P, P, 1, 0, res, None) == \
        _lib.EIK_ERR_ARG
    ok = (ctypes.c_int64 * 2)(9, 7)
    for hh, hb in ((float("inf"), 0.1), (0.1, float("inf")), (float("nan"), 0.1),
                   (0.1, float("nan")), (-0.1, 0.1), (0.1, 0.0)):
        assert lib.eik_residual_noalloc(2, ok, hh, hb, P, P, P, 1, 0, res, None) == \
            _lib.EIK_ERR_ARG, (hh, hb)


def test_fft_series_validates_arguments_without_gpu(lib):
    """eik_fft_series rejects bad sizes, spacings, term counts and f~ before
    any CUDA call."""
    import math
    from paper_1403_1937_gb300 import _lib
    P = ctypes.c_void_p(0x1000)      # never dereferenced: the checks fail first
    d = (ctypes.c_int64 * 2)(9, 7)
    ft = ctypes.c_double()
    for dims in ((1, 7), (9, 1), (3601, 8), (8, 3601)):
        dd = (ctypes.c_int64 * 2)(*dims)
        assert lib.eik_fft_series(dd, 0.1, 0.1, P, P, 1, 2, 0.0, P, None, ctypes.byref(ft),
                                  None) == _lib.EIK_ERR_ARG, dims
    for h, hb in ((0.0, 0.1), (0.1, -1.0), (math.inf, 0.1), (0.1, math.nan)):
        assert lib.eik_fft_series(d, h, hb, P, P, 1, 2, 0.0, P, None, None, None) == \
            _lib.EIK_ERR_ARG, (h, hb)
    for terms, fti, nsrc in ((-1, 0.0, 1), (65, 0.0, 1), (2, -1.0, 1), (2, math.inf, 1),
                             (2, 0.0, 0)):
        assert lib.eik_fft_series(d, 0.1, 0.1, P, P, nsrc, terms, fti, P, None, None,
                                  None) == _lib.EIK_ERR_ARG, (terms, fti, nsrc)
    assert lib.eik_fft_series(d, 0.1, 0.1, None, P, 1, 2, 0.0, P, None, None, None) == \
        _lib.EIK_ERR_ARG
    assert lib.eik_fft_series(d, 0.1, 0.1, P, P, 1, 2, 0.0, None, None, None, None) == \
        _lib.EIK_ERR_ARG
