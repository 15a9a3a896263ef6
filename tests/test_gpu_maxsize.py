"""The largest tree the library accepts (N = 2^30 - 1 points, where the child
index 2n + 2 still fits int32): the tree is a permutation of the points,
sampled kNN and ball results equal brute force, the ablation kernels agree,
and a query count of 2^32 is rejected before any device access."""
import ctypes
import math

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_MAX = (1 << 30) - 1


@pytest.fixture(scope="module")
def kdt():
    from paper_2210_12859_gb300 import build

    build.build_library()
    from paper_2210_12859_gb300 import kdt as k

    return k


def test_largest_tree(kdt):
    # seeded uniform points made on the device (12.9 GB; the peak of this test
    # is about 60 GB of device memory)
    g = torch.Generator(device="cuda")
    g.manual_seed(221012859)
    pts = torch.rand((N_MAX, 3), generator=g, device="cuda", dtype=torch.float32)
    qs = torch.rand((1 << 16, 3), generator=g, device="cuda", dtype=torch.float32)
    tree = kdt.kdt_build(pts)
    coords, ids = kdt.kdt_tree_export(tree)
    srt, _ = torch.sort(ids)
    assert torch.equal(srt, torch.arange(N_MAX, dtype=torch.int32, device="cuda"))
    del srt
    assert torch.equal(coords, pts[ids.long()])
    root = int(ids[0].item())
    del coords, ids
    # the root is the point of rank L(N) in (x, index) order (the median rule)
    order = torch.sort(pts[:, 0].contiguous(), stable=True).indices
    assert int(order[oracle.left_size(N_MAX)].item()) == root
    del order
    ki, kd = kdt.kdt_knn(tree, qs, 8, flags=kdt.KDT_MORTON)
    kdt.kdt_status(tree)
    for fl in (kdt.KDT_PLAIN_STEP, kdt.KDT_STACK, kdt.KDT_CLOSE_FIRST):
        ai, ad = kdt.kdt_knn(tree, qs, 8, flags=fl | kdt.KDT_MORTON)
        assert torch.equal(ai, ki) and torch.equal(ad.view(torch.int32), kd.view(torch.int32))
    counts = kdt.kdt_radius_count(tree, qs, 0.002)
    pts_h = pts.cpu().numpy()
    qs_h = qs.cpu().numpy()
    del pts
    sample = np.random.default_rng(3).choice(len(qs_h), 12, replace=False)
    wi, wd = oracle.knn_brute_threaded(pts_h, qs_h[sample], 8)
    assert np.array_equal(ki.cpu().numpy()[sample], wi)
    assert np.array_equal(kd.cpu().numpy()[sample].view(np.uint32), wd.view(np.uint32))
    wc, _, _, _ = oracle.radius_brute(pts_h, qs_h[sample[:3]], 0.002)
    assert np.array_equal(counts.cpu().numpy()[sample[:3]], wc)


def test_query_count_limit(kdt):
    """Q >= 2^32 is rejected on the host (dummy pointers are never read)."""
    tree = kdt.kdt_build(torch.rand((100, 3), device="cuda"))
    lib = kdt._lib
    d = ctypes.c_void_p(256)
    rc = lib.kdt_knn(tree.handle, d, 1 << 32, 8, ctypes.c_float(math.inf), 0, d, d, None)
    assert rc == kdt.KDT_EINVAL
    rc = lib.kdt_radius_count(tree.handle, d, 1 << 32, ctypes.c_float(0.1), 0, d, None)
    assert rc == kdt.KDT_EINVAL
