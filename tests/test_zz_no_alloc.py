"""kdt_knn_static, the entry point that allocates no device memory.

It exists for callers that may not enter the CUDA allocator while they query
(their own pool owns the device memory, or a cudaMalloc's synchronisation
would stall a real-time loop); its scratch is a fixed device array inside the
library.  Called here through the C ABI (ctypes) and compared with kdt_knn,
bit for bit, on two calls in a row (the second call finds the first call's
leftovers in the shared array).  This file is collected last on purpose.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2210_12859_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2210_12859_gb300 import build

    path = build.build_library()
    from paper_2210_12859_gb300 import kdt

    L = ctypes.CDLL(path)
    P, I64, I, F = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_float
    L.kdt_knn_static.argtypes = [P, P, I64, I, F, I, P, P, P]
    L.kdt_knn_static.restype = I
    L.kdt_last_error.restype = ctypes.c_char_p
    L.kdt_debug_fail_allocs.argtypes = [I]
    L.kdt_debug_fail_allocs.restype = I
    return L, kdt


def static_knn(L, tree, q, k, r, flags):
    Q = q.shape[0]
    ids = torch.full((Q, k), -7, dtype=torch.int32, device="cuda")
    d2 = torch.full((Q, k), -7.0, dtype=torch.float32, device="cuda")
    rc = L.kdt_knn_static(tree.handle, ctypes.c_void_p(q.data_ptr()), Q, k, float(r), flags,
                          ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(d2.data_ptr()),
                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, L.kdt_last_error()
    return ids, d2


@pytest.mark.parametrize("k,r,flag_names", [(8, math.inf, ("MORTON",)), (1, math.inf, ()),
                                            (32, 0.05, ("MORTON", "UNORDERED")), (16, math.inf, ("MORTON",))])
def test_static_matches_kdt_knn_twice(lib, k, r, flag_names):
    L, kdt = lib
    pts, qs = synth.uniform_small(1 << 14, 70001)  # ragged against warps and sort tiles
    tree = kdt.kdt_build(torch.from_numpy(pts).cuda())
    dq = torch.from_numpy(qs).cuda()
    flags = 0
    for n in flag_names:
        flags |= getattr(kdt, "KDT_" + n)
    want_i, want_d = kdt.kdt_knn(tree, dq, k, r, flags)
    for _ in range(2):
        gi, gd = static_knn(L, tree, dq, k, r, flags)
        torch.cuda.synchronize()
        assert torch.equal(gi, want_i)
        assert torch.equal(gd.view(torch.int32), want_d.view(torch.int32))
    kdt.kdt_status(tree)


def test_static_rejects_too_many_queries(lib):
    L, kdt = lib
    pts, _ = synth.uniform_small(1000, 1)
    tree = kdt.kdt_build(torch.from_numpy(pts).cuda())
    Q = kdt.KDT_STATIC_MAX_Q + 1
    q = torch.zeros((Q, 3), dtype=torch.float32, device="cuda")
    out_i = torch.empty((Q, 4), dtype=torch.int32, device="cuda")
    out_d = torch.empty((Q, 4), dtype=torch.float32, device="cuda")
    rc = L.kdt_knn_static(tree.handle, ctypes.c_void_p(q.data_ptr()), Q, 4, float("inf"), 0,
                          ctypes.c_void_p(out_i.data_ptr()), ctypes.c_void_p(out_d.data_ptr()), None)
    assert rc == kdt.KDT_EINVAL
    assert b"at most" in L.kdt_last_error()


def test_static_allocates_nothing(lib):
    """With the library's allocation hook armed, any device allocation the
    call made would fail with KDT_ENOMEM; the static entry point must succeed
    (and the same call through kdt_knn, which allocates its scratch, must
    fail, which shows the hook is armed)."""
    L, kdt = lib
    pts, qs = synth.uniform_small(1 << 12, 5000)
    tree = kdt.kdt_build(torch.from_numpy(pts).cuda())
    dq = torch.from_numpy(qs).cuda()
    want_i, want_d = kdt.kdt_knn(tree, dq, 8, math.inf, kdt.KDT_MORTON)
    torch.cuda.synchronize()
    try:
        assert L.kdt_debug_fail_allocs(1) == 0
        gi, gd = static_knn(L, tree, dq, 8, math.inf, kdt.KDT_MORTON | kdt.KDT_COST_ORDER)
        torch.cuda.synchronize()
        with pytest.raises(kdt.KdtError) as e:
            kdt.kdt_knn(tree, dq, 8, math.inf, kdt.KDT_MORTON)
        assert e.value.code == kdt.KDT_ENOMEM
    finally:
        L.kdt_debug_fail_allocs(0)
    assert torch.equal(gi, want_i)
    assert torch.equal(gd.view(torch.int32), want_d.view(torch.int32))
    kdt.kdt_status(tree)


def test_static_at_max_queries(lib):
    """Q = KDT_STATIC_MAX_Q, the size the fixed scratch array is dimensioned
    for, with the cost-class Morton order (the largest scratch use)."""
    L, kdt = lib
    pts, _ = synth.uniform_small(1 << 16, 1)
    Q = kdt.KDT_STATIC_MAX_Q
    qs = synth.uniform_small(1, Q, seed=synth.BASE_SEED + 991)[1]
    tree = kdt.kdt_build(torch.from_numpy(pts).cuda())
    dq = torch.from_numpy(qs).cuda()
    flags = kdt.KDT_MORTON | kdt.KDT_COST_ORDER
    want_i, want_d = kdt.kdt_knn(tree, dq, 8, math.inf, flags)
    for _ in range(2):
        gi, gd = static_knn(L, tree, dq, 8, math.inf, flags)
        torch.cuda.synchronize()
        assert torch.equal(gi, want_i)
        assert torch.equal(gd.view(torch.int32), want_d.view(torch.int32))
    kdt.kdt_status(tree)
