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


def header_constants():
    """Enumerator values of include/sw_cgne.h (NAME = value inside enum blocks)."""
    src = open(os.path.join(ROOT, "include", "sw_cgne.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for body in re.findall(r"enum\s*\w*\s*\{(.*?)\}", src, flags=re.S):
        for name, val in re.findall(r"\b(SW_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
            out[name] = int(val)
    return out


def test_binding_constants_match_the_header():
    import paper_1312_3265_gb300._binding as bd
    consts = header_constants()
    assert "SW_SITE_SHAPES" in consts and "SW_PARAM_SITE_BLOCKING" in consts
    for name, val in consts.items():
        if hasattr(bd, name):
            assert getattr(bd, name) == val, name
    for name in ("SW_PARAM_CHUNK", "SW_PARAM_RELIABLE_DELTA", "SW_PARAM_RELIABLE_DELTA_F16", "SW_PARAM_NS_SW",
                 "SW_PARAM_NS_WILSON", "SW_PARAM_GRAPHS", "SW_PARAM_SITE_BLOCKING", "SW_PARAM_GROUP_FAST",
                 "SW_PARAM_PERSISTENT", "SW_PARAM_WILSON_LEAN", "SW_SITE_SHAPES", "SW_PREC_F64", "SW_PREC_F32_RELIABLE", "SW_PREC_F16_RELIABLE"):
        assert getattr(bd, name) == consts[name], name


def test_tunable_ranges(lib):
    """sw_set_param accepts exactly the documented values (host-side state, no
    GPU needed) and sw_get_param returns them."""
    import paper_1312_3265_gb300._binding as bd
    lib.sw_set_param.argtypes = [ctypes.c_int, ctypes.c_double]
    lib.sw_get_param.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    cases = {
        bd.SW_PARAM_CHUNK: ([1, 4, 4096], [0, 4097, -1]),
        bd.SW_PARAM_RELIABLE_DELTA: ([1e-6, 0.5], [0.0, 1.0, -1e-3]),
        bd.SW_PARAM_RELIABLE_DELTA_F16: ([1e-3], [0.0, 2.0]),
        bd.SW_PARAM_NS_SW: ([1, 2, 4], [0, 3, 8]),
        bd.SW_PARAM_NS_WILSON: ([1, 2, 4], [0, 3, 8]),
        bd.SW_PARAM_GRAPHS: ([0, 1], [2, -1]),
        bd.SW_PARAM_GROUP_FAST: ([0, 1], [2]),
        bd.SW_PARAM_PERSISTENT: ([0, 1], [2, 0.5]),
        bd.SW_PARAM_WILSON_LEAN: ([-1, 0, 1], [2, -2, 0.5]),
        bd.SW_PARAM_SITE_BLOCKING: (list(range(bd.SW_SITE_SHAPES)), [-1, bd.SW_SITE_SHAPES, 1.5]),
    }
    v = ctypes.c_double()
    for key, (good, bad) in cases.items():
        assert lib.sw_get_param(key, ctypes.byref(v)) == 0
        old = v.value
        try:
            for g in good:
                assert lib.sw_set_param(key, g) == 0, (key, g)
                assert lib.sw_get_param(key, ctypes.byref(v)) == 0 and v.value == g
            for b in bad:
                assert lib.sw_set_param(key, b) < 0, (key, b)
                assert lib.sw_get_param(key, ctypes.byref(v)) == 0 and v.value == good[-1]  # unchanged
        finally:
            assert lib.sw_set_param(key, old) == 0
    assert lib.sw_set_param(12345, 1.0) < 0
    assert lib.sw_get_param(12345, ctypes.byref(v)) < 0
