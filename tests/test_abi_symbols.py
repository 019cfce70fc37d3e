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
