"""GPU parity of the builder and the plain traversal against the CPU oracle.

Bar: bit-exact tree arrays, neighbour ids and FP32 squared distances; visit
counts of the ordered and unordered state machines equal to the oracle's.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2210_12859_gb300 import synth
from kdt_checks import check_tree

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


def assert_same(gi, gd, wi, wd):
    gi = gi.cpu().numpy()
    gd = gd.cpu().numpy()
    assert np.array_equal(gi, wi), f"ids differ at {np.argwhere(gi != wi)[:5].tolist()}"
    assert np.array_equal(bits(gd), bits(wd)), "squared distances differ"


# ---------------------------------------------------------------- builder

BUILD_CASES = [(1, 3), (2, 3), (3, 2), (6, 2), (7, 3), (8, 3), (31, 1), (33, 4), (100, 5), (255, 3), (256, 3),
               (257, 3), (1000, 8), (2047, 2), (2049, 6), (5000, 7), (40000, 3), (65537, 4)]


@pytest.mark.parametrize("N,D", BUILD_CASES)
def test_build_equals_oracle_tree(kdt, N, D):
    g = np.random.default_rng(N * 10 + D)
    if N % 2:
        pts = g.integers(0, 7, size=(N, D)).astype(np.float32)  # heavy ties
    else:
        pts = g.standard_normal((N, D)).astype(np.float32)
    tree = kdt.kdt_build(cu(pts))
    coords, ids = kdt.kdt_tree_export(tree)
    want = oracle.build(pts)
    assert np.array_equal(ids.cpu().numpy(), want)
    assert np.array_equal(bits(coords.cpu().numpy()), bits(pts[want]))


def test_build_six_point_example(kdt):
    pts = np.array([[2, 3], [5, 4], [9, 6], [4, 7], [8, 1], [7, 2]], dtype=np.float32)
    tree = kdt.kdt_build(cu(pts))
    _, ids = kdt.kdt_tree_export(tree)
    assert ids.cpu().tolist() == [5, 1, 2, 0, 3, 4]


def test_build_signed_zeros(kdt):
    pts = np.array([[0.0, 1.0], [-0.0, 1.0], [0.0, -0.0], [-0.0, 0.0], [1.0, 2.0]] * 7, dtype=np.float32)
    tree = kdt.kdt_build(cu(pts))
    _, ids = kdt.kdt_tree_export(tree)
    assert np.array_equal(ids.cpu().numpy(), oracle.build(pts))


def test_rebuild_reuses_tree(kdt):
    a, _ = synth.uniform_small(3000, 1)
    b = synth.uniform(3000, 3, seed=5)
    tree = kdt.kdt_build(cu(a))
    kdt.kdt_rebuild(tree, cu(b))
    _, ids = kdt.kdt_tree_export(tree)
    assert np.array_equal(ids.cpu().numpy(), oracle.build(b))


def test_tree_save_load_roundtrip(kdt, tmp_path):
    pts, qs = synth.uniform_small(5000, 2000)
    tree = kdt.kdt_build(cu(pts))
    path = str(tmp_path / "tree.kdt")
    kdt.kdt_tree_save(tree, path)
    back = kdt.kdt_tree_load(path)
    a, b = kdt.kdt_tree_export(tree), kdt.kdt_tree_export(back)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    ra = kdt.kdt_knn(tree, cu(qs), 8, flags=kdt.KDT_MORTON)
    rb = kdt.kdt_knn(back, cu(qs), 8, flags=kdt.KDT_MORTON)
    assert torch.equal(ra[0], rb[0]) and torch.equal(ra[1], rb[1])
    raw = bytearray(open(path, "rb").read())
    raw[100] ^= 1
    open(path, "wb").write(bytes(raw))
    with pytest.raises(kdt.KdtError) as e:
        kdt.kdt_tree_load(path)
    assert e.value.code == kdt.KDT_EIO


def test_build_rejects_bad_input(kdt):
    pts = np.zeros((10, 3), dtype=np.float32)
    pts[4, 2] = np.inf
    with pytest.raises(kdt.KdtError) as e:
        kdt.kdt_build(cu(pts))
    assert e.value.code == kdt.KDT_ENONFINITE
    with pytest.raises(kdt.KdtError) as e:
        kdt.kdt_build(cu(np.zeros((4, 9), dtype=np.float32)))
    assert e.value.code == kdt.KDT_EINVAL
    with pytest.raises(kdt.KdtError):
        kdt.kdt_build(cu(np.zeros((0, 3), dtype=np.float32)))
    # asynchronous build reports the same failure through kdt_status
    tree = kdt.kdt_build(cu(pts), opts=kdt.KDT_BUILD_ASYNC)
    with pytest.raises(kdt.KdtError) as e:
        kdt.kdt_status(tree)
    assert e.value.code == kdt.KDT_ENONFINITE
    kdt.kdt_status(tree)  # cleared


# ---------------------------------------------------------------- queries

@pytest.fixture(scope="module")
def small(kdt):
    """Uniform 3-D, N = Q = 2^14, queries in [-0.1, 1.1]^3."""
    pts, qs = synth.uniform_small()
    tree = kdt.kdt_build(cu(pts))
    return pts, qs, tree, cu(qs), oracle.build(pts)


@pytest.mark.parametrize("flags_name", ["ORDERED", "UNORDERED", "MORTON", "NO_STAGE", "UNORDERED|MORTON",
                                        "MORTON|COST_ORDER"])
@pytest.mark.parametrize("k", [1, 8])
def test_small_uniform_bit_exact(kdt, small, flags_name, k):
    pts, qs, tree, dq, _ = small
    flags = 0
    for f in flags_name.split("|"):
        flags |= getattr(kdt, "KDT_" + f)
    wi, wd = oracle.knn_brute(pts, qs, k)
    if k == 1:
        gi, gd = kdt.kdt_fcp(tree, dq, flags=flags)
        assert_same(gi, gd, wi[:, 0], wd[:, 0])
    else:
        gi, gd = kdt.kdt_knn(tree, dq, k, flags=flags)
        assert_same(gi, gd, wi, wd)
    kdt.kdt_status(tree)


@pytest.mark.parametrize("ordered", [True, False])
@pytest.mark.parametrize("k,r", [(8, math.inf), (1, math.inf), (16, 0.05), (3, 0.0)])
def test_visit_counts_equal_oracle(kdt, small, ordered, k, r):
    pts, qs, tree, dq, node_pid = small
    sub = slice(0, 4096)
    _, _, nv = oracle.knn_tree(pts, node_pid, qs[sub], k, r, ordered)
    flags = 0 if ordered else kdt.KDT_UNORDERED
    v = kdt.kdt_knn_visits(tree, dq[sub].contiguous(), k, r, flags)
    assert np.array_equal(v.cpu().numpy(), nv)


@pytest.mark.parametrize("k", [2, 3, 5, 13, 16, 17, 32, 64])
@pytest.mark.parametrize("r", [math.inf, 0.04])
def test_k_sweep(kdt, small, k, r):
    pts, qs, tree, dq, _ = small
    sub = slice(0, 2048)
    wi, wd = oracle.knn_brute(pts, qs[sub], k, r)
    gi, gd = kdt.kdt_knn(tree, dq[sub].contiguous(), k, r, flags=kdt.KDT_MORTON)
    assert_same(gi, gd, wi, wd)


@pytest.mark.parametrize("D", [1, 2, 3, 4, 5, 8])
@pytest.mark.parametrize("k", [1, 8, 16, 40])
def test_dimensions(kdt, D, k):
    pts = synth.uniform(6000, D, seed=D)
    qs = synth.uniform(700, D, -0.1, 1.1, seed=D + 100)
    tree = kdt.kdt_build(cu(pts))
    wi, wd = oracle.knn_brute(pts, qs, k)
    for flags in (0, kdt.KDT_UNORDERED | kdt.KDT_MORTON):
        gi, gd = kdt.kdt_knn(tree, cu(qs), k, flags=flags)
        assert_same(gi, gd, wi, wd)


def test_edge_cases(kdt):
    # N = 1
    p1 = np.array([[0.5, 0.5, 0.5]], dtype=np.float32)
    t1 = kdt.kdt_build(cu(p1))
    q = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]], dtype=np.float32)
    gi, gd = kdt.kdt_knn(t1, cu(q), 4)
    wi, wd = oracle.knn_brute(p1, q, 4)
    assert_same(gi, gd, wi, wd)
    # duplicates, k > N, zero radius, far queries
    g = np.random.default_rng(3)
    pts = g.integers(0, 3, size=(500, 3)).astype(np.float32)
    qs = np.concatenate([pts[:50], g.integers(-2, 5, size=(50, 3)).astype(np.float32), np.full((3, 3), 1e20, np.float32)])
    t = kdt.kdt_build(cu(pts))
    for k, r in [(64, math.inf), (64, 0.0), (10, 1.0), (1, 0.0), (7, 3e19)]:
        wi, wd = oracle.knn_brute(pts, qs, k, r)
        gi, gd = kdt.kdt_knn(t, cu(qs), k, r)
        assert_same(gi, gd, wi, wd)
    # k > N: every point, then empty slots
    few = pts[:37].copy()
    tf = kdt.kdt_build(cu(few))
    for k in (37, 40, 64):
        wi, wd = oracle.knn_brute(few, qs, k)
        gi, gd = kdt.kdt_knn(tf, cu(qs), k)
        assert_same(gi, gd, wi, wd)
    # Q = 0 is a no-op
    kdt.kdt_knn(t, cu(np.zeros((0, 3), np.float32)), 5)
    kdt.kdt_status(t)


def test_query_rejects_bad_arguments(kdt, small):
    _, _, tree, dq, _ = small
    for k, r in [(0, 1.0), (65, 1.0), (4, -1.0), (4, math.nan)]:
        with pytest.raises(kdt.KdtError) as e:
            kdt.kdt_knn(tree, dq[:10].contiguous(), k, r)
        assert e.value.code == kdt.KDT_EINVAL
    with pytest.raises(kdt.KdtError) as e:
        kdt.kdt_knn(tree, dq[:10].contiguous(), 4, flags=kdt.KDT_LEARNED)
    assert e.value.code == kdt.KDT_ENOMODEL


def test_host_entry_point(kdt):
    pts, qs = synth.uniform_small(5000, 3000)
    ids = np.empty((3000, 8), np.int32)
    d2 = np.empty((3000, 8), np.float32)
    kdt.kdt_knn_host(pts, qs, 8, out_ids=ids, out_d2=d2, flags=kdt.KDT_MORTON)
    wi, wd = oracle.knn_brute(pts, qs, 8)
    assert np.array_equal(ids, wi) and np.array_equal(bits(d2), bits(wd))


@pytest.mark.parametrize("k", [8, 5])
@pytest.mark.parametrize("pin", ["all", "queries", "outputs", "none", "unaligned"])
def test_host_entry_point_in_place(kdt, pin, k):
    """Page-locked query and result buffers are used in place (the kernels
    read and write host memory); pageable ones are copied; a result buffer
    off a 16-byte boundary takes the word stores.  Same results each way."""
    pts, qs = synth.uniform_small(6000, 2500)
    pq = torch.from_numpy(qs)
    if pin in ("all", "queries"):
        pq = pq.pin_memory()
    pinned_out = pin in ("all", "outputs", "unaligned")
    ids = torch.empty(2500 * k + 1, dtype=torch.int32)
    d2 = torch.empty(2500 * k + 1, dtype=torch.float32)
    if pinned_out:
        ids, d2 = ids.pin_memory(), d2.pin_memory()
    o = 1 if pin == "unaligned" else 0
    oi, od = ids[o:o + 2500 * k].view(2500, k), d2[o:o + 2500 * k].view(2500, k)
    kdt.kdt_knn_host(pts, pq, k, out_ids=oi, out_d2=od, flags=kdt.KDT_MORTON)
    wi, wd = oracle.knn_brute(pts, qs, k)
    assert np.array_equal(oi.numpy(), wi) and np.array_equal(bits(od.numpy()), bits(wd))


def test_fp64_cross_check(kdt, small):
    pts, qs, tree, dq, _ = small
    sub = slice(0, 1024)
    gi, gd = kdt.kdt_knn(tree, dq[sub].contiguous(), 8)
    i64, d64 = oracle.knn_brute_f64(pts, qs[sub], 8)
    gd = gd.cpu().numpy().astype(np.float64)
    # each FP32 term fl(fl(p - q)^2) is within 3u of exact and two additions
    # of non-negative terms add 2u: |d2 - exact| <= 5u d2 (u = 2^-24); allow 16u
    assert np.allclose(gd, d64, rtol=8 * 2.0 ** -23, atol=1e-30)
    assert (gi.cpu().numpy() == i64).mean() > 0.999


# ---------------------------------------------------------------- full size

@pytest.fixture(scope="module")
def gmm_full(kdt):
    """64-component Gaussian mixture, N = Q = 2^24 (the large clustered workload)."""
    pts, qs = synth.gmm_large()
    dp, dq = cu(pts), cu(qs)
    tree = kdt.kdt_build(dp)
    return pts, qs, tree, dq


def test_full_size_tree_property(kdt, gmm_full):
    pts, _, tree, _ = gmm_full
    coords, ids = kdt.kdt_tree_export(tree)
    check_tree(pts, ids.cpu().numpy(), coords.cpu().numpy())


def test_full_size_bench_configuration(kdt, gmm_full):
    """The launch the benchmark times (all 2^24 queries, k = 8, Morton order),
    checked on sampled outputs."""
    pts, qs, tree, dq = gmm_full
    gi, gd = kdt.kdt_knn(tree, dq, 8, flags=kdt.KDT_MORTON | kdt.KDT_COST_ORDER)
    kdt.kdt_status(tree)
    sample = np.random.default_rng(8).choice(len(qs), size=192, replace=False)
    wi, wd = oracle.knn_brute_threaded(pts, qs[sample], 8)
    sel = torch.from_numpy(sample).cuda()
    assert_same(gi[sel], gd[sel], wi, wd)


@pytest.mark.parametrize("k,r,flags_name", [(1, math.inf, "MORTON"), (64, math.inf, "MORTON"),
                                            (8, 0.005, "MORTON"), (8, math.inf, "UNORDERED|MORTON"),
                                            (16, math.inf, "ORDERED")])
def test_full_size_tree_query_subsets(kdt, gmm_full, k, r, flags_name):
    """Variants on the full 2^24 tree with a 2^16-query subset (sampled outputs)."""
    pts, qs, tree, dq = gmm_full
    flags = 0
    for f in flags_name.split("|"):
        flags |= getattr(kdt, "KDT_" + f)
    sub = np.sort(np.random.default_rng(k + 1).choice(len(qs), size=1 << 16, replace=False))
    q = cu(qs[sub])
    gi, gd = kdt.kdt_knn(tree, q, k, r, flags=flags)
    kdt.kdt_status(tree)
    sample = np.random.default_rng(k).choice(len(sub), size=96, replace=False)
    wi, wd = oracle.knn_brute_threaded(pts, qs[sub][sample], k, r)
    sel = torch.from_numpy(sample).cuda()
    assert_same(gi[sel], gd[sel], wi, wd)
