"""The C-ABI library loads and exports every entry point include/kdt.h
declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "kdt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(kdt_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2210_12859_gb300 import build

    return ctypes.CDLL(build.build_library())


def test_header_declares_entry_points():
    names = _declared()
    for n in ("kdt_build", "kdt_knn", "kdt_fcp", "kdt_free", "kdt_last_error", "kdt_build_batched",
              "kdt_knn_batched", "kdt_radius_model_train"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_names_match_abi():
    from paper_2210_12859_gb300 import kdt

    missing = [n for n in _declared() if not hasattr(kdt, n)]
    assert not missing, f"no Python binding for: {missing}"


def test_last_error_callable_without_gpu(lib):
    lib.kdt_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.kdt_last_error(), bytes)
