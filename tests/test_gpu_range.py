"""GPU parity of the range queries (ball: every point within a radius; box:
every point inside [lo, hi]) against the oracle: counts and offsets exact,
hits equal to the brute-force sets and, in order, to the oracle's stack-free
range traversal; squared distances bit-exact; every node layout (D = 1..8,
stored split dimensions), with and without Morton order."""
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


def same_sets(off, ids, want_off, want_ids, d2=None, want_d2=None):
    """Per query, the hits as (id, d2 bits) sets; the oracle lists ids in index order."""
    assert np.array_equal(off, want_off)
    for q in range(len(off) - 1):
        a, b = off[q], off[q + 1]
        order = np.argsort(ids[a:b], kind="stable")
        assert np.array_equal(ids[a:b][order], want_ids[a:b]), q
        if d2 is not None:
            assert np.array_equal(bits(d2[a:b][order]), bits(want_d2[a:b])), q


def radius_for(pts, hits):
    """A radius that holds about `hits` points around a typical point."""
    N, D = pts.shape
    ext = np.prod(pts.max(0) - pts.min(0) + 1e-6)
    from math import gamma, pi

    unit = pi ** (D / 2) / gamma(D / 2 + 1)
    return float((hits * ext / (N * unit)) ** (1.0 / D))


CASES = [(1, 5000, 0), (2, 6000, 0), (3, 20000, 0), (4, 8000, 0), (5, 4000, 0), (8, 3000, 0), (3, 20000, 1),
         (2, 5000, 1)]


def build(kdt, pts, widest):
    return kdt.kdt_build(cu(pts), opts=kdt.KDT_BUILD_WIDEST if widest else 0)


def oracle_tree(pts, widest):
    if widest:
        return oracle.build_widest(pts)
    return oracle.build(pts), None


@pytest.mark.parametrize("D,N,widest", CASES)
def test_radius_equals_brute(kdt, D, N, widest):
    g = np.random.default_rng(10 * D + N + widest)
    pts = synth.uniform(N, D, seed=D + N)
    qs = np.concatenate([pts[g.integers(0, N, 100)], g.random((157, D)).astype(np.float32)])
    r = radius_for(pts, 20)
    tree = build(kdt, pts, widest)
    counts, want_off, want_ids, want_d2 = oracle.radius_brute(pts, qs, r)
    assert want_off[-1] > 5 * len(qs)
    pid, dims = oracle_tree(pts, widest)
    _, t_off, t_ids, t_d2 = oracle.range_tree(pts, pid, qs, radius=r, node_dim=dims)
    for flags in (0, kdt.KDT_MORTON):
        off, ids, d2 = kdt.kdt_radius_search(tree, cu(qs), r, flags=flags)
        kdt.kdt_status(tree)
        off, ids, d2 = off.cpu().numpy(), ids.cpu().numpy(), d2.cpu().numpy()
        same_sets(off, ids, want_off, want_ids, d2, want_d2)
        # the same hits in the same order as the oracle's stack-free range traversal
        assert np.array_equal(ids, t_ids) and np.array_equal(bits(d2), bits(t_d2))
        assert np.array_equal(kdt.kdt_radius_count(tree, cu(qs), r, flags).cpu().numpy(), counts)


@pytest.mark.parametrize("D,N,widest", CASES)
def test_box_equals_brute(kdt, D, N, widest):
    g = np.random.default_rng(7 * D + N + widest)
    pts = synth.uniform(N, D, seed=D * N)
    Q = 211
    centre = g.random((Q, D)).astype(np.float32)
    half = (g.random((Q, D)) * 2 * radius_for(pts, 16)).astype(np.float32)
    lo, hi = centre - half, centre + half
    lo[:5] = pts[:5]  # boxes whose faces pass through points (inclusive bounds)
    hi[:5] = pts[:5]
    lo[5] = hi[5] + 0.1  # an empty box
    tree = build(kdt, pts, widest)
    _, want_off, want_ids = oracle.box_brute(pts, lo, hi)
    assert want_off[-1] > 3 * Q
    pid, dims = oracle_tree(pts, widest)
    _, _, t_ids, _ = oracle.range_tree(pts, pid, lo, hi, node_dim=dims)
    for flags in (0, kdt.KDT_MORTON):
        off, ids = kdt.kdt_box_search(tree, cu(lo), cu(hi), flags=flags)
        kdt.kdt_status(tree)
        off, ids = off.cpu().numpy(), ids.cpu().numpy()
        same_sets(off, ids, want_off, want_ids)
        assert np.array_equal(ids, t_ids)


def test_duplicates_and_zero_radius(kdt):
    g = np.random.default_rng(3)
    pts = g.integers(0, 4, size=(3000, 3)).astype(np.float32)  # 64 distinct sites, ~47 copies each
    qs = np.concatenate([pts[:50], pts[:50] + np.float32(0.5)])
    tree = kdt.kdt_build(cu(pts))
    for r in (0.0, 1.0, 1.5):
        off, ids, d2 = kdt.kdt_radius_search(tree, cu(qs), r)
        _, want_off, want_ids, want_d2 = oracle.radius_brute(pts, qs, r)
        same_sets(off.cpu().numpy(), ids.cpu().numpy(), want_off, want_ids, d2.cpu().numpy(), want_d2)
    off, ids = kdt.kdt_box_search(tree, cu(pts[:40]), cu(pts[:40] + 1))
    _, want_off, want_ids = oracle.box_brute(pts, pts[:40], pts[:40] + 1)
    same_sets(off.cpu().numpy(), ids.cpu().numpy(), want_off, want_ids)


@pytest.mark.parametrize("N", [1, 2, 3, 7, 100])
def test_small_trees_infinite_range(kdt, N):
    pts = synth.uniform(N, 3, seed=N)
    qs = synth.uniform(9, 3, seed=N + 1)
    tree = kdt.kdt_build(cu(pts))
    off, ids, d2 = kdt.kdt_radius_search(tree, cu(qs), float("inf"))
    _, want_off, want_ids, want_d2 = oracle.radius_brute(pts, qs, float("inf"))
    assert want_off[-1] == 9 * N
    same_sets(off.cpu().numpy(), ids.cpu().numpy(), want_off, want_ids, d2.cpu().numpy(), want_d2)
    lo = np.full((4, 3), -np.inf, np.float32)
    hi = np.full((4, 3), np.inf, np.float32)
    off, ids = kdt.kdt_box_search(tree, cu(lo), cu(hi))
    assert np.array_equal(off.cpu().numpy(), np.arange(5) * N)


def test_empty_queries_and_bad_arguments(kdt):
    pts = synth.uniform(100, 3, seed=1)
    tree = kdt.kdt_build(cu(pts))
    qs = torch.empty((0, 3), dtype=torch.float32, device="cuda")
    off, ids, d2 = kdt.kdt_radius_search(tree, qs, 0.1)
    assert off.cpu().tolist() == [0] and ids.numel() == 0
    off, ids = kdt.kdt_box_search(tree, qs, qs)
    assert off.cpu().tolist() == [0] and ids.numel() == 0
    with pytest.raises(kdt.KdtError):
        kdt.kdt_radius_count(tree, cu(pts[:4]), -1.0)
    with pytest.raises(kdt.KdtError):
        kdt.kdt_radius_count(tree, cu(pts[:4]), float("nan"))
    with pytest.raises(kdt.KdtError):
        kdt.kdt_radius_count(tree, cu(pts[:4]), 0.1, flags=kdt.KDT_UNORDERED)


def test_fill_with_mismatched_offsets_is_reported(kdt):
    pts = synth.uniform(1000, 3, seed=2)
    qs = pts[:64]
    tree = kdt.kdt_build(cu(pts))
    r = radius_for(pts, 10)
    counts = kdt.kdt_radius_count(tree, cu(qs), r)
    assert int(counts.min()) >= 1
    zero = torch.zeros(65, dtype=torch.int64, device="cuda")  # every slice empty: nothing may be written
    ids, _ = kdt.kdt_radius_fill(tree, cu(qs), r, zero, 0, with_d2=False)
    with pytest.raises(kdt.KdtError):
        kdt.kdt_status(tree)
    kdt.kdt_status(tree)  # the recorded state was cleared


def test_fill_is_deterministic_and_matches_knn(kdt):
    mix = synth.gmm_mixture(16, 3, 0.02, 5)
    pts = synth.gmm_sample(mix, 50000, 6)
    qs = synth.gmm_sample(mix, 2000, 7)
    tree = kdt.kdt_build(cu(pts))
    r = 0.004
    off, ids, d2 = kdt.kdt_radius_search(tree, cu(qs), r)
    off2, ids2, d22 = kdt.kdt_radius_search(tree, cu(qs), r)
    assert torch.equal(ids, ids2) and torch.equal(off, off2) and torch.equal(d2, d22)
    # the k best of the ball (by (d2, id)) are the radius-bounded kNN result
    k = 8
    kid, kd2 = kdt.kdt_knn(tree, cu(qs), k, max_radius=r)
    off, ids, d2 = off.cpu().numpy(), ids.cpu().numpy(), d2.cpu().numpy()
    kid, kd2 = kid.cpu().numpy(), kd2.cpu().numpy()
    for q in range(len(qs)):
        a, b = off[q], off[q + 1]
        order = np.lexsort((ids[a:b], d2[a:b]))[:k]
        m = len(order)
        assert np.array_equal(ids[a:b][order], kid[q, :m]), q
        assert np.array_equal(bits(d2[a:b][order]), bits(kd2[q, :m])), q
        assert np.all(kid[q, m:] == -1)


@pytest.mark.parametrize("kind", ["ball", "box"])
def test_fill_vector_and_word_paths_agree(kdt, kind):
    """The fill pass writes 16-byte groups into aligned outputs and single
    words otherwise (here: outputs one word past a 16-byte boundary).  Both
    give the oracle machine's hits in traversal order, over slices of every
    start alignment and length (0 to dozens of hits)."""
    import ctypes

    mix = synth.gmm_mixture(16, 3, 0.02, 8)
    pts = synth.gmm_sample(mix, 40000, 9)
    qs = np.concatenate([synth.gmm_sample(mix, 3000, 10), synth.uniform(200, 3, seed=11)])
    tree = kdt.kdt_build(cu(pts))
    dq = cu(qs)
    r = 0.005
    lo, hi = (dq - r).contiguous(), (dq + r).contiguous()
    counts = kdt.kdt_radius_count(tree, dq, r) if kind == "ball" else kdt.kdt_box_count(tree, lo, hi)
    off, total = kdt.kdt_offsets(counts)
    assert total > 0
    res = []
    for shift in (0, 1):
        ids = torch.full((total + 8,), -5, dtype=torch.int32, device="cuda")
        d2 = torch.full((total + 8,), -5.0, dtype=torch.float32, device="cuda")
        pi, pd = ids.data_ptr() + 4 * shift, d2.data_ptr() + 4 * shift
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        if kind == "ball":
            rc = kdt._lib.kdt_radius_fill(tree.handle, ctypes.c_void_p(dq.data_ptr()), len(qs), ctypes.c_float(r), 0,
                                          ctypes.c_void_p(off.data_ptr()), ctypes.c_void_p(pi), ctypes.c_void_p(pd),
                                          stream)
        else:
            rc = kdt._lib.kdt_box_fill(tree.handle, ctypes.c_void_p(lo.data_ptr()), ctypes.c_void_p(hi.data_ptr()),
                                       len(qs), 0, ctypes.c_void_p(off.data_ptr()), ctypes.c_void_p(pi), stream)
        assert rc == 0
        torch.cuda.synchronize()
        kdt.kdt_status(tree)
        ids, d2 = ids.cpu().numpy(), d2.cpu().numpy()
        # nothing outside the written range was touched
        assert (ids[:shift] == -5).all() and (ids[shift + total:] == -5).all()
        res.append((ids[shift:shift + total], d2[shift:shift + total]))
    assert np.array_equal(res[0][0], res[1][0])
    if kind == "ball":
        assert np.array_equal(bits(res[0][1]), bits(res[1][1]))
    node_pid = oracle.build(pts)
    if kind == "ball":
        _, woff, wids, wd2 = oracle.range_tree(pts, node_pid, qs, radius=r)
        assert np.array_equal(bits(res[0][1]), bits(wd2))
    else:
        _, woff, wids = oracle.range_tree(pts, node_pid, qs - np.float32(r), qs + np.float32(r))[:3]
    assert np.array_equal(off.cpu().numpy(), woff) and np.array_equal(res[0][0], wids)


def test_full_size_sampled(kdt):
    """2^22 clustered points, 2^18 queries: counts and sampled hit sets equal brute force."""
    mix = synth.gmm_mixture(64, 3, 0.01, 11)
    pts = synth.gmm_sample(mix, 1 << 22, 12)
    qs = synth.gmm_sample(mix, 1 << 18, 13)
    tree = kdt.kdt_build(cu(pts))
    r = 0.002
    dq = cu(qs)
    off, ids, d2 = kdt.kdt_radius_search(tree, dq, r, flags=kdt.KDT_MORTON)
    kdt.kdt_status(tree)
    off, ids, d2 = off.cpu().numpy(), ids.cpu().numpy(), d2.cpu().numpy()
    sample = np.random.default_rng(0).choice(len(qs), 96, replace=False)
    _, want_off, want_ids, want_d2 = oracle.radius_brute(pts, qs[sample], r)
    for j, q in enumerate(sample):
        a, b = off[q], off[q + 1]
        wa, wb = want_off[j], want_off[j + 1]
        order = np.argsort(ids[a:b], kind="stable")
        assert np.array_equal(ids[a:b][order], want_ids[wa:wb]), q
        assert np.array_equal(bits(d2[a:b][order]), bits(want_d2[wa:wb])), q
    assert off[-1] > len(qs)


@pytest.mark.parametrize("D,N,widest", [(3, 20000, 0), (2, 5000, 1), (4, 8000, 0), (6, 3000, 0)])
def test_range_visits_equal_oracle(kdt, D, N, widest):
    """KDT_RANGE_VISITS: the count calls report processed nodes, equal to the
    oracle's range traversal, for balls and boxes."""
    g = np.random.default_rng(D + N)
    pts = synth.uniform(N, D, seed=D * 3 + N)
    qs = (g.random((200, D)) * 1.2 - 0.1).astype(np.float32)
    r = radius_for(pts, 15)
    tree = build(kdt, pts, widest)
    pid, dims = oracle_tree(pts, widest)
    for flags in (kdt.KDT_RANGE_VISITS, kdt.KDT_RANGE_VISITS | kdt.KDT_MORTON):
        v = kdt.kdt_radius_count(tree, cu(qs), r, flags).cpu().numpy()
        assert np.array_equal(v, oracle.range_visits(pts, pid, qs, radius=r, node_dim=dims))
        lo, hi = qs - np.float32(r), qs + np.float32(r)
        vb = kdt.kdt_box_count(tree, cu(lo), cu(hi), flags).cpu().numpy()
        assert np.array_equal(vb, oracle.range_visits(pts, pid, lo, hi, node_dim=dims))
    with pytest.raises(kdt.KdtError):
        kdt.kdt_radius_fill(tree, cu(qs), r, torch.zeros(201, dtype=torch.int64, device="cuda"), 0,
                            flags=kdt.KDT_RANGE_VISITS)
