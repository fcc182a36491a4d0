"""The C-ABI library builds, loads and exports every symbol include/ams.h
declares (no compute calls: these run without a GPU)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ams.h")


@pytest.fixture(scope="module")
def built_lib():
    from paper_2606_04864_gb300._build import build
    path = build()
    return ctypes.CDLL(path)


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(ams_[a-z_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["ams_setup", "ams_setup_batched", "ams_solve", "ams_solve_adjoint", "ams_destroy",
                     "ams_status_string", "ams_last_error", "ams_options_default"]:
        assert required in names


def test_every_declared_symbol_is_exported(built_lib):
    missing = [n for n in _declared_functions() if not hasattr(built_lib, n)]
    assert not missing, missing


def test_checking_build_exports_the_same_boundary(built_lib):
    """The AMS_DEBUG variant (device-side index checks) builds from the same
    sources and exports every declared symbol, ams_debug_selftest included."""
    from paper_2606_04864_gb300._build import build
    dbg = ctypes.CDLL(build(debug=True))
    missing = [n for n in _declared_functions() if not hasattr(dbg, n)]
    assert not missing, missing
    assert hasattr(built_lib, "ams_debug_selftest") and hasattr(dbg, "ams_debug_selftest")


def test_python_binding_covers_every_symbol():
    from paper_2606_04864_gb300._lib import SIGNATURES
    assert sorted(SIGNATURES) == _declared_functions()


def test_status_strings_without_gpu(built_lib):
    f = built_lib.ams_status_string
    f.restype = ctypes.c_char_p
    f.argtypes = [ctypes.c_int]
    assert f(0) == b"AMS_OK"
    assert f(2) == b"AMS_ERR_NOT_SPD"
    assert f(99) == b"AMS_ERR_UNKNOWN"


def test_options_default_without_gpu(built_lib):
    from paper_2606_04864_gb300._lib import ams_options
    o = ams_options()
    fn = built_lib.ams_options_default
    fn.argtypes = [ctypes.POINTER(ams_options)]
    fn.restype = None
    fn(ctypes.byref(o))
    assert o.precision == 2 and o.maxit == 10000 and o.coarse == 1 and o.cg_variant == -1


def test_destroy_null_is_ok(built_lib):
    fn = built_lib.ams_destroy
    fn.argtypes = [ctypes.c_void_p]
    fn.restype = ctypes.c_int
    assert fn(None) == 0


def test_product_path_has_no_cpu_fallback(monkeypatch, tmp_path):
    """The binding refuses to run when the library is missing."""
    import paper_2606_04864_gb300._lib as L
    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(L, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        L.lib()


def test_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2606_04864_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                src = open(os.path.join(dirpath, fn), errors="replace").read()
                assert "import oracle" not in src and "from oracle" not in src, fn
