"""GPU parity of the payload reductions (sum, mean, photon-map density) over
ball hits (summed in traversal order inside the range kernel) and over kNN
results (summed in list order), bit-exact against the oracle."""
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


def same_bits(a, b):
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    nan = np.isnan(a) & np.isnan(b)
    return np.array_equal(np.where(nan, 0, a.view(np.uint32)), np.where(nan, 0, b.view(np.uint32)))


MODES = (0, 1, 2)


@pytest.mark.parametrize("D,N,C,widest,r", [(3, 20000, 3, 0, 0.08), (2, 5000, 1, 0, 0.08), (4, 6000, 6, 0, 0.25),
                                            (7, 3000, 8, 0, 0.45), (3, 20000, 4, 1, 0.08)])
def test_radius_reduce_equals_oracle(kdt, D, N, C, widest, r):
    g = np.random.default_rng(D * 100 + C)
    pts = synth.uniform(N, D, seed=D + C)
    pay = g.standard_normal((N, C)).astype(np.float32)
    qs = np.concatenate([pts[:64], g.random((100, D)).astype(np.float32)])
    if widest:
        pid, dims = oracle.build_widest(pts)
        tree = kdt.kdt_build(cu(pts), opts=kdt.KDT_BUILD_WIDEST)
    else:
        pid, dims = oracle.build(pts), None
        tree = kdt.kdt_build(cu(pts))
    kdt.kdt_tree_set_payload(tree, cu(pay))
    for mode in MODES:
        want, wc = oracle.range_reduce(pts, pid, qs, r, pay, mode, node_dim=dims)
        assert wc.mean() > 3
        for flags in (0, kdt.KDT_MORTON):
            out, cnt = kdt.kdt_radius_reduce(tree, cu(qs), r, mode, flags, with_counts=True)
            kdt.kdt_status(tree)
            assert np.array_equal(cnt.cpu().numpy(), wc)
            assert same_bits(out.cpu().numpy(), want), (mode, flags)


@pytest.mark.parametrize("k,r", [(1, np.inf), (8, np.inf), (32, np.inf), (16, 0.02), (64, 0.05)])
def test_knn_reduce_equals_oracle(kdt, k, r):
    mix = synth.gmm_mixture(16, 3, 0.02, 3)
    pts = synth.gmm_sample(mix, 30000, 4)
    qs = synth.gmm_queries(mix, 500, 0.2, 5)
    g = np.random.default_rng(k)
    power = g.random((len(pts), 3)).astype(np.float32)  # photon power (RGB)
    tree = kdt.kdt_build(cu(pts))
    kdt.kdt_tree_set_payload(tree, cu(power))
    ki, kd = oracle.knn_brute(pts, qs, k, r)
    for mode in MODES:
        want = oracle.knn_reduce(ki, kd, power, mode)
        for flags in (0, kdt.KDT_MORTON, kdt.KDT_UNORDERED):
            out = kdt.kdt_knn_reduce(tree, cu(qs), k, r, mode, flags)
            assert same_bits(out.cpu().numpy(), want), (mode, flags)


def test_payload_layouts_and_rebuild(kdt):
    """Payload permutation into node order on every layout; a rebuild drops it."""
    for D in (3, 4, 6):
        pts = synth.uniform(4000, D, seed=D)
        pay = np.arange(4000 * 2, dtype=np.float32).reshape(4000, 2)
        tree = kdt.kdt_build(cu(pts))
        kdt.kdt_tree_set_payload(tree, cu(pay))
        qs = pts[:50]
        # r = 0: each query's only hit is itself (distinct points): the payload comes back
        out = kdt.kdt_radius_reduce(tree, cu(qs), 0.0, kdt.KDT_REDUCE_SUM).cpu().numpy()
        assert np.array_equal(out, pay[:50])
        out = kdt.kdt_knn_reduce(tree, cu(qs), 1, mode=kdt.KDT_REDUCE_SUM).cpu().numpy()
        assert np.array_equal(out, pay[:50])
        kdt.kdt_rebuild(tree, cu(pts))
        with pytest.raises(kdt.KdtError):
            kdt.kdt_radius_reduce(tree, cu(qs), 0.1)


def test_reduce_edge_cases(kdt):
    pts = synth.uniform(500, 3, seed=8)
    tree = kdt.kdt_build(cu(pts))
    with pytest.raises(kdt.KdtError):
        kdt.kdt_knn_reduce(tree, cu(pts[:3]), 4)  # no payload yet
    with pytest.raises(kdt.KdtError):
        kdt.kdt_tree_set_payload(tree, cu(np.zeros((500, 9), np.float32)))  # C > 8
    pay = np.ones((500, 1), np.float32)
    kdt.kdt_tree_set_payload(tree, cu(pay))
    far = np.full((4, 3), 50.0, np.float32)  # no hit within the radius: 0 in every mode
    for mode in MODES:
        out = kdt.kdt_radius_reduce(tree, cu(far), 0.1, mode).cpu().numpy()
        assert not out.any()
        out = kdt.kdt_knn_reduce(tree, cu(far), 8, 0.1, mode).cpu().numpy()
        assert not out.any()
    with pytest.raises(kdt.KdtError):
        kdt.kdt_radius_reduce(tree, cu(far), 0.1, 3)
    # duplicates at distance 0: density divides by pi * 0 (IEEE: +inf), as the oracle
    dup = np.repeat(pts[:1], 20, axis=0)
    t2 = kdt.kdt_build(cu(dup))
    kdt.kdt_tree_set_payload(t2, cu(np.ones((20, 1), np.float32)))
    out = kdt.kdt_knn_reduce(t2, cu(dup[:2]), 4, mode=kdt.KDT_REDUCE_DENSITY).cpu().numpy()
    ki, kd = oracle.knn_brute(dup, dup[:2], 4)
    assert same_bits(out, oracle.knn_reduce(ki, kd, np.ones((20, 1), np.float32), kdt.KDT_REDUCE_DENSITY))
    assert np.all(np.isinf(out))
