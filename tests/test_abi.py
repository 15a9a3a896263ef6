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


def test_tuning_file_round_trip_without_gpu(lib, tmp_path):
    """Tuning files are host-only: rows written before the claim / inline
    fields existed load with the defaults, new rows keep their values, and
    malformed rows are rejected with KDT_EIO (-7)."""
    import json

    lib.kdt_tuning_load.argtypes = [ctypes.c_char_p]
    lib.kdt_tuning_save.argtypes = [ctypes.c_char_p]
    src = tmp_path / "in.json"
    src.write_text('[\n'
                   '  {"gpu": "cpu-test-a", "D": 3, "k_bucket": 3, "log2n": 18, "stage_levels": 4},\n'
                   '  {"gpu": "cpu-test-b", "D": 2, "k_bucket": 0, "log2n": 20, "stage_levels": 0, '
                   '"claim_steps": 128, "inline_depth": 0, "light_run": 8}\n]\n')
    assert lib.kdt_tuning_load(str(src).encode()) == 0
    out = tmp_path / "out.json"
    assert lib.kdt_tuning_save(str(out).encode()) == 0
    rows = {r["gpu"]: r for r in json.loads(out.read_text())}
    assert rows["cpu-test-a"]["stage_levels"] == 4
    assert rows["cpu-test-a"]["claim_steps"] == 64 and rows["cpu-test-a"]["inline_depth"] == 2
    assert rows["cpu-test-b"]["claim_steps"] == 128 and rows["cpu-test-b"]["inline_depth"] == 0
    assert rows["cpu-test-b"]["light_run"] == 8 and rows["cpu-test-a"]["light_run"] == 1
    for bad in ('"stage_levels": 99}', '"stage_levels": 0, "claim_steps": 0}', '"stage_levels": 0, "light_run": 0}',
                '"stage_levels": 0, "claim_steps": 64, "inline_depth": 5}'):
        src.write_text('[\n  {"gpu": "x", "D": 3, "k_bucket": 3, "log2n": 18, ' + bad + '\n]\n')
        assert lib.kdt_tuning_load(str(src).encode()) == -7
    assert lib.kdt_tuning_load(str(tmp_path / "missing.json").encode()) == -7


def test_size_limits_rejected_on_the_host(lib):
    """N must be in [1, 2^30) and D in [1, 8]: checked before any device
    access, so a dummy pointer is never touched."""
    lib.kdt_build_ex.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                 ctypes.POINTER(ctypes.c_void_p)]
    out = ctypes.c_void_p()
    dummy = ctypes.c_void_p(16)
    for n, d in (((1 << 30), 3), (0, 3), (-5, 3), (100, 0), (100, 9)):
        assert lib.kdt_build_ex(dummy, n, d, 0, None, ctypes.byref(out)) == -1, (n, d)
        assert not out.value
    assert lib.kdt_build_ex(None, 100, 3, 0, None, ctypes.byref(out)) == -1


def test_injected_allocation_failure_without_gpu(lib):
    """kdt_debug_fail_allocs makes a build fail with KDT_ENOMEM (-3) before any
    device access; the hook counts down and clears."""
    lib.kdt_debug_fail_allocs.argtypes = [ctypes.c_int]
    lib.kdt_build_ex.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                 ctypes.POINTER(ctypes.c_void_p)]
    out = ctypes.c_void_p()
    assert lib.kdt_debug_fail_allocs(1) == 0
    assert lib.kdt_build_ex(ctypes.c_void_p(16), 100, 3, 0, None, ctypes.byref(out)) == -3
    assert not out.value
    assert lib.kdt_debug_fail_allocs(-1) == -1
    assert lib.kdt_debug_fail_allocs(0) == 0


def test_binding_rejects_host_tensors_no_cpu_fallback():
    """The product path has no CPU fallback: host tensors are refused before
    any library call."""
    torch = pytest.importorskip("torch")
    from paper_2210_12859_gb300 import kdt

    pts = torch.rand((64, 3))
    with pytest.raises(TypeError):
        kdt.kdt_build(pts)
    with pytest.raises(TypeError):
        kdt.kdt_offsets(torch.zeros(4, dtype=torch.int32))


def test_binding_without_library_raises(tmp_path):
    """Importing the binding where libkdt.so is missing raises ImportError."""
    import importlib.util
    import shutil

    pytest.importorskip("torch")
    src = os.path.join(ROOT, "paper_2210_12859_gb300", "kdt.py")
    shutil.copy(src, tmp_path / "kdt_copy.py")
    spec = importlib.util.spec_from_file_location("kdt_copy", tmp_path / "kdt_copy.py")
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError):
        spec.loader.exec_module(mod)


def test_host_entry_outputs_are_written_in_place_or_rejected():
    """kdt_knn_host writes into the caller's arrays: an output of the wrong
    dtype, layout or shape is rejected before the call (a converted copy would
    receive the results and drop them)."""
    import numpy as np

    from paper_2210_12859_gb300 import kdt

    pts = np.zeros((16, 3), np.float32)
    qs = np.zeros((4, 3), np.float32)
    good_i, good_d = np.empty((4, 2), np.int32), np.empty((4, 2), np.float32)
    with pytest.raises(TypeError):
        kdt.kdt_knn_host(pts, qs, 2, out_ids=np.empty((4, 2), np.int64), out_d2=good_d)
    with pytest.raises(TypeError):
        kdt.kdt_knn_host(pts, qs, 2, out_ids=good_i, out_d2=np.empty((2, 4), np.float32).T)
    with pytest.raises(ValueError):
        kdt.kdt_knn_host(pts, qs, 2, out_ids=np.empty((4, 3), np.int32), out_d2=good_d)
    with pytest.raises(ValueError):
        kdt.kdt_knn_host(pts, np.zeros((4, 2), np.float32), 2, out_ids=good_i, out_d2=good_d)
