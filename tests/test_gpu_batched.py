"""GPU parity of the batched forest path: every tree equals the oracle's tree
of its cloud, every query's kNN equals the oracle's brute force over its own
cloud, for the single persistent (graph-replayed) launch and for one launch
per tree."""
import math

import numpy as np
import pytest

import oracle
from paper_2210_12859_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kdt():
    from paper_2210_12859_gb300 import build

    build.build_library()
    from paper_2210_12859_gb300 import kdt as k

    return k


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def bits(x):
    return np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)


@pytest.fixture(scope="module")
def forest(kdt):
    c = synth.clouds(60, 3.0, 12.0, seed=11)
    # add empty clouds and a single-point cloud in the middle
    sizes = list(np.diff(c.offsets))
    pts = [c.points[c.offsets[i]:c.offsets[i + 1]] for i in range(60)]
    qs = [c.queries[c.qoffsets[i]:c.qoffsets[i + 1]] for i in range(60)]
    pts.insert(7, np.zeros((0, 3), np.float32))
    qs.insert(7, np.zeros((0, 3), np.float32))
    pts.insert(20, np.array([[0.5, 0.5, 0.5]], np.float32))
    qs.insert(20, np.random.default_rng(1).random((9, 3)).astype(np.float32))
    pts.insert(30, np.zeros((0, 3), np.float32))
    qs.insert(30, np.random.default_rng(2).random((5, 3)).astype(np.float32))  # queries, no points
    off = np.concatenate([[0], np.cumsum([len(p) for p in pts])]).astype(np.int64)
    qoff = np.concatenate([[0], np.cumsum([len(q) for q in qs])]).astype(np.int64)
    P = np.concatenate(pts).astype(np.float32)
    Q = np.concatenate(qs).astype(np.float32)
    f = kdt.kdt_build_batched(cu(P), off)
    return pts, qs, P, Q, off, qoff, f


def test_forest_trees_equal_oracle(kdt, forest):
    pts, qs, P, Q, off, qoff, f = forest
    coords, ids = kdt.kdt_forest_export(f)
    coords, ids = coords.cpu().numpy(), ids.cpu().numpy()
    for i, p in enumerate(pts):
        if len(p) == 0:
            continue
        want = oracle.build(p)
        assert np.array_equal(ids[off[i]:off[i + 1]], want), i
        assert np.array_equal(bits(coords[off[i]:off[i + 1]]), bits(p[want]))


@pytest.mark.parametrize("flags_name", ["ORDERED", "MORTON", "PER_TREE", "UNORDERED|MORTON"])
@pytest.mark.parametrize("k,r", [(8, math.inf), (3, 0.05), (20, math.inf)])
def test_forest_knn_equals_oracle(kdt, forest, flags_name, k, r):
    pts, qs, P, Q, off, qoff, f = forest
    flags = 0
    for n in flags_name.split("|"):
        flags |= getattr(kdt, "KDT_" + n)
    dq = cu(Q)
    for rep in range(2):  # the second call replays the captured graph
        gi, gd = kdt.kdt_knn_batched(f, dq, qoff, k, r, flags=flags)
        gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
        for i, (p, q) in enumerate(zip(pts, qs)):
            if len(q) == 0:
                continue
            if len(p) == 0:
                assert (gi[qoff[i]:qoff[i + 1]] == -1).all() and np.isinf(gd[qoff[i]:qoff[i + 1]]).all()
                continue
            wi, wd = oracle.knn_brute(p, q, k, r)
            assert np.array_equal(gi[qoff[i]:qoff[i + 1]], wi), i
            assert np.array_equal(bits(gd[qoff[i]:qoff[i + 1]]), bits(wd)), i


@pytest.mark.parametrize("k,r,unordered", [(8, math.inf, False), (3, 0.05, True), (20, math.inf, False)])
def test_forest_visits_equal_oracle(kdt, forest, k, r, unordered):
    """Processed nodes of every forest query equal the oracle machine's on
    that cloud's own tree (0 for queries of an empty cloud)."""
    pts, qs, P, Q, off, qoff, f = forest
    flags = kdt.KDT_UNORDERED if unordered else 0
    v = kdt.kdt_knn_batched_visits(f, cu(Q), qoff, k, r, flags).cpu().numpy()
    for i, (p, q) in enumerate(zip(pts, qs)):
        if len(q) == 0:
            continue
        if len(p) == 0:
            assert (v[qoff[i]:qoff[i + 1]] == 0).all()
            continue
        _, _, wv = oracle.knn_tree(p, oracle.build(p), q, k, r, ordered=not unordered)
        assert np.array_equal(v[qoff[i]:qoff[i + 1]], wv), i


def test_forest_graph_recaptures_on_new_arguments(kdt, forest):
    pts, qs, P, Q, off, qoff, f = forest
    dq = cu(Q)
    a = kdt.kdt_knn_batched(f, dq, qoff, 8)
    dq2 = dq.clone()
    b = kdt.kdt_knn_batched(f, dq2, qoff, 8)
    c = kdt.kdt_knn_batched(f, dq2, qoff, 4)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert torch.equal(c[0], b[0][:, :4])


def test_forest_matches_single_tree_builds(kdt):
    c = synth.clouds(8, 10.0, 14.0, seed=3)
    f = kdt.kdt_build_batched(cu(c.points), c.offsets)
    gi, gd = kdt.kdt_knn_batched(f, cu(c.queries), c.qoffsets, 8, flags=kdt.KDT_MORTON)
    for i in range(8):
        t = kdt.kdt_build(cu(c.points[c.offsets[i]:c.offsets[i + 1]]))
        si, sd = kdt.kdt_knn(t, cu(c.queries[c.qoffsets[i]:c.qoffsets[i + 1]]), 8)
        assert torch.equal(si, gi[c.qoffsets[i]:c.qoffsets[i + 1]])
        assert torch.equal(sd, gd[c.qoffsets[i]:c.qoffsets[i + 1]])


@pytest.mark.parametrize("k", [1, 8, 32])
def test_forest_launch_parameters_do_not_change_results(kdt, forest, k):
    pts, qs, P, Q, off, qoff, f = forest
    dq = cu(Q)
    ref_i, ref_d = kdt.kdt_knn_batched(f, dq, qoff, k, flags=kdt.KDT_PER_TREE)
    for threads, inl, lr in ((0, 0, 0), (32, 1, 4), (64, 2, 8), (128, 1, 1)):
        for cs in (0, 1, 16, 256):
            kdt.kdt_forest_set_launch(f, threads, cs, inl, lr)
            for flags in (kdt.KDT_MORTON, 0):
                gi, gd = kdt.kdt_knn_batched(f, dq, qoff, k, flags=flags)
                assert torch.equal(gi, ref_i) and torch.equal(gd.view(torch.int32), ref_d.view(torch.int32))
    kdt.kdt_forest_set_launch(f, 0, 0)
    for bad in ((96 + 64, 0), (48, 0), (0, 257), (-32, 0), (0, 0, 3), (0, 0, 0, 65)):
        with pytest.raises(kdt.KdtError):
            kdt.kdt_forest_set_launch(f, *bad)


def test_forest_autotune(kdt, forest):
    pts, qs, P, Q, off, qoff, f = forest
    dq = cu(Q)
    ref_i, ref_d = kdt.kdt_knn_batched(f, dq, qoff, 8, flags=kdt.KDT_PER_TREE)
    th, cs, il, lr, ms = kdt.kdt_forest_autotune(f, dq, qoff, 8, flags=kdt.KDT_MORTON)
    assert th in (64, 128) and cs in (16, 32, 64, 128) and il in (1, 2) and lr in (1, 4, 8) and ms > 0
    gi, gd = kdt.kdt_knn_batched(f, dq, qoff, 8, flags=kdt.KDT_MORTON)
    assert torch.equal(gi, ref_i) and torch.equal(gd.view(torch.int32), ref_d.view(torch.int32))
    with pytest.raises(kdt.KdtError):
        kdt.kdt_forest_autotune(f, dq, qoff, 8, flags=kdt.KDT_PER_TREE)
    kdt.kdt_forest_set_launch(f, 0, 0)
