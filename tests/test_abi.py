"""The C-ABI library builds, loads and exports every symbol include/*.h declares
(no compute calls: these run without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M):
            name = m.group(1)
            if name not in ("if", "sizeof", "return"):
                names.append(name)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1312_3265_gb300 import build as b
    path = b.lib_path()
    if not os.path.exists(path):
        b.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("sw_hypercube_build", "sw_dslash_apply", "wilson_dslash_apply", "cgne_solve",
                 "sw_status_string"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    lib.sw_status_string.restype = ctypes.c_char_p
    assert lib.sw_status_string(0) == b"ok"
    assert b"aligned" in lib.sw_status_string(-3)
    assert lib.sw_status_string(12345) == b"unknown status"
    lib.sw_last_cuda_error.restype = ctypes.c_char_p
    assert lib.sw_last_cuda_error() == b"cudaSuccess"


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_1312_3265_gb300._binding as bd
    monkeypatch.setattr(bd, "_lib", None)
    monkeypatch.setattr(bd, "_lib_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        bd.lib()
