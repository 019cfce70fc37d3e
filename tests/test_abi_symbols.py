"""The C ABI library builds, loads and exports every entry point that
include/dec.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dec.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dec_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2104_05999_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_path_entry_points():
    names = _declared()
    for n in ("dec_create", "dec_destroy", "dec_last_error", "dec_mesh_upload",
              "dec_hodge_assemble", "dec_laplacian_build", "dec_solve",
              "dec_k_eff"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_the_header():
    from paper_2104_05999_gb300 import abi
    names = set(_declared()) - {"dec_last_error"}
    assert names <= set(abi.SIGNATURES)


def test_binding_refuses_wrong_dtypes():
    import numpy as np
    from paper_2104_05999_gb300.abi import _ptr
    with pytest.raises(TypeError):
        _ptr(np.zeros(3, dtype=np.float32), np.float64)
    with pytest.raises(TypeError):
        _ptr(np.zeros((3, 4), dtype=np.float64)[:, 1], np.float64)


def _prototypes():
    src = open(os.path.join(ROOT, "include", "dec.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for name, params in re.findall(r"\b(dec_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src):
        params = " ".join(params.split())
        out[name] = [] if params in ("", "void") else [p.strip() for p in params.split(",")]
    return out


def test_binding_argument_types_match_the_header():
    # pointer <-> c_void_p, int32_t <-> c_int32, int64_t <-> c_int64,
    # double <-> c_double, int <-> c_int: a wrong width would pass garbage
    from paper_2104_05999_gb300 import abi
    protos = _prototypes()
    assert set(abi.SIGNATURES) <= set(protos)
    for name, argt in abi.SIGNATURES.items():
        params = protos[name]
        assert len(params) == len(argt), name
        for p, t in zip(params, argt):
            if "*" in p:
                assert t is ctypes.c_void_p or issubclass(t, ctypes._Pointer), (name, p, t)
                continue
            if p.startswith("int32_t"):
                want = ctypes.c_int32
            elif p.startswith("int64_t"):
                want = ctypes.c_int64
            elif p.startswith("double"):
                want = ctypes.c_double
            elif p.startswith("int "):
                want = ctypes.c_int
            else:
                raise AssertionError(f"{name}: unhandled parameter type {p!r}")
            assert t is want, (name, p, t)
