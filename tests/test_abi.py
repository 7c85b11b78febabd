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
