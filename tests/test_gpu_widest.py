"""GPU parity of trees with a stored per-node split dimension (widest extent,
KDT_BUILD_WIDEST): tree arrays and dimensions equal to the oracle's, results
equal to brute force, visit counts equal to the oracle's traversal."""
import math

import numpy as np
import pytest

import oracle
from paper_2210_12859_gb300 import synth
from kdt_checks import check_tree_widest

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


@pytest.mark.parametrize("N,D", [(1, 3), (2, 2), (6, 2), (7, 3), (100, 1), (257, 3), (1000, 2), (4097, 3), (50000, 3)])
def test_widest_tree_equals_oracle(kdt, N, D):
    g = np.random.default_rng(N + D)
    pts = (g.random((N, D)) * np.array([1.0, 0.3, 2.0][:D])).astype(np.float32)
    if N % 2:
        pts = g.integers(0, 6, size=(N, D)).astype(np.float32)
    tree = kdt.kdt_build(cu(pts), opts=kdt.KDT_BUILD_WIDEST)
    coords, ids = kdt.kdt_tree_export(tree)
    dims = kdt.kdt_tree_split_dims(tree)
    want_ids, want_dims = oracle.build_widest(pts)
    assert np.array_equal(ids.cpu().numpy(), want_ids)
    assert np.array_equal(dims.cpu().numpy(), want_dims)
    assert np.array_equal(bits(coords.cpu().numpy()), bits(pts[want_ids]))


def test_round_robin_dims_reported(kdt):
    pts = synth.uniform(100, 3, seed=1)
    tree = kdt.kdt_build(cu(pts))
    dims = kdt.kdt_tree_split_dims(tree).cpu().numpy()
    assert np.array_equal(dims, np.floor(np.log2(np.arange(100) + 1)).astype(int) % 3)


@pytest.fixture(scope="module")
def clustered(kdt):
    mix = synth.gmm_mixture(16, 3, 0.02, 5)
    pts = synth.gmm_sample(mix, 20000, 6)
    qs = synth.gmm_queries(mix, 3000, 0.1, 7)
    tree = kdt.kdt_build(cu(pts), opts=kdt.KDT_BUILD_WIDEST)
    ids, dims = oracle.build_widest(pts)
    return pts, qs, tree, ids, dims


@pytest.mark.parametrize("k,r", [(1, math.inf), (8, math.inf), (16, 0.05), (40, math.inf)])
@pytest.mark.parametrize("flags_name", ["ORDERED", "UNORDERED", "MORTON", "MORTON|COST_ORDER"])
def test_widest_queries_equal_brute(kdt, clustered, k, r, flags_name):
    pts, qs, tree, _, _ = clustered
    flags = 0
    for n in flags_name.split("|"):
        flags |= getattr(kdt, "KDT_" + n)
    gi, gd = kdt.kdt_knn(tree, cu(qs), k, r, flags=flags)
    wi, wd = oracle.knn_brute(pts, qs, k, r)
    assert np.array_equal(gi.cpu().numpy(), wi)
    assert np.array_equal(bits(gd.cpu().numpy()), bits(wd))
    kdt.kdt_status(tree)


@pytest.mark.parametrize("ordered", [True, False])
@pytest.mark.parametrize("k", [1, 8])
def test_widest_visit_counts_equal_oracle(kdt, clustered, ordered, k):
    pts, qs, tree, ids, dims = clustered
    _, _, nv = oracle.knn_tree_dims(pts, ids, dims, qs, k, math.inf, ordered)
    v = kdt.kdt_knn_visits(tree, cu(qs), k, flags=0 if ordered else kdt.KDT_UNORDERED)
    assert np.array_equal(v.cpu().numpy(), nv)


def test_widest_learned_save_load_rebuild(kdt, clustered, tmp_path):
    pts, qs, tree, ids, dims = clustered
    kdt.kdt_radius_model_train(tree, cu(qs[:2000]), 8, epochs=4, seed=2)
    a = kdt.kdt_knn(tree, cu(qs), 8, flags=kdt.KDT_MORTON)
    b = kdt.kdt_knn(tree, cu(qs), 8, flags=kdt.KDT_MORTON | kdt.KDT_LEARNED)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    path = str(tmp_path / "widest.kdt")
    kdt.kdt_tree_save(tree, path)
    back = kdt.kdt_tree_load(path)
    assert torch.equal(kdt.kdt_tree_split_dims(back), kdt.kdt_tree_split_dims(tree))
    c = kdt.kdt_knn(back, cu(qs), 8)
    assert torch.equal(a[0], c[0]) and torch.equal(a[1], c[1])
    other = synth.uniform(len(pts), 3, seed=9)
    kdt.kdt_rebuild(back, cu(other))
    want_ids, want_dims = oracle.build_widest(other)
    assert np.array_equal(kdt.kdt_tree_export(back)[1].cpu().numpy(), want_ids)
    assert np.array_equal(kdt.kdt_tree_split_dims(back).cpu().numpy(), want_dims)


def test_widest_rejects_high_dimension(kdt):
    with pytest.raises(kdt.KdtError) as e:
        kdt.kdt_build(cu(synth.uniform(100, 4, seed=1)), opts=kdt.KDT_BUILD_WIDEST)
    assert e.value.code == kdt.KDT_EINVAL


def test_widest_full_size(kdt):
    """The large clustered workload (N = Q = 2^24) on a widest-extent tree:
    the tree property at full size and sampled queries against brute force."""
    pts, qs = synth.gmm_large()
    tree = kdt.kdt_build(cu(pts), opts=kdt.KDT_BUILD_WIDEST)
    _, ids = kdt.kdt_tree_export(tree)
    check_tree_widest(pts, ids.cpu().numpy(), kdt.kdt_tree_split_dims(tree).cpu().numpy())
    sub = np.sort(np.random.default_rng(3).choice(len(qs), size=1 << 16, replace=False))
    gi, gd = kdt.kdt_knn(tree, cu(qs[sub]), 8, flags=kdt.KDT_MORTON | kdt.KDT_COST_ORDER)
    sample = np.random.default_rng(4).choice(len(sub), size=96, replace=False)
    wi, wd = oracle.knn_brute_threaded(pts, qs[sub][sample], 8)
    assert np.array_equal(gi.cpu().numpy()[sample], wi)
    assert np.array_equal(bits(gd.cpu().numpy()[sample]), bits(wd))
