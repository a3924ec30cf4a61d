"""The C-ABI library builds, loads and exports every declared entry point (CPU only)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(fmm_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2005_12351_gb300 import build
    return build.build()


def test_every_declared_symbol_is_exported(libpath):
    lib = ctypes.CDLL(libpath)
    names = declared_functions()
    assert len(names) >= 13
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.fmm_status_string.restype = ctypes.c_char_p
    assert lib.fmm_status_string(0) == b"ok"
    assert lib.fmm_status_string(-6) == b"device memory budget exceeded"


def test_binding_refuses_missing_library(monkeypatch, tmp_path):
    """No CPU fallback: a missing extension is an import-time error."""
    pytest.importorskip("torch")
    from paper_2005_12351_gb300 import fmm
    monkeypatch.setattr(fmm, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(fmm, "_lib", None)
    with pytest.raises(ImportError):
        fmm.lib()


def test_create_tree_reports_missing_device(libpath):
    """On a machine without a GPU the library returns a status, it does not abort."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    lib = ctypes.CDLL(libpath)
    h = ctypes.c_void_p()
    st = lib.fmm_create_tree(ctypes.byref(h), 0, None, 64, 0, ctypes.c_size_t(0))
    assert st == -1 and not h.value


def test_server_create_without_gpu_returns_status(libpath):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    lib = ctypes.CDLL(libpath)
    h = ctypes.c_void_p()
    st = lib.fmm_server_create(ctypes.byref(h), 0, 2, 0, ctypes.c_size_t(0))
    assert st != 0 and not h.value
