"""Pins for the CPU oracle (no GPU).

Each test checks the oracle against something other than itself: the worked
example of the paper's Figure 1, closed forms, library routines (numpy sorting
and searching, torch's bfloat16 conversion), independent brute force and the
invariants the paper states (Sec. 3.1: the state machine visits the same nodes
in the same order as the recursion).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2210_12859_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "six_point_2d.json")


# ---------------------------------------------------------------- topology

def _subtree_size_by_ancestry(n: int, root: int) -> int:
    """Count nodes of an n-node level-order tree having `root` as ancestor
    (or being it), by walking parent links (n-1)//2 ... independently of any
    size formula."""
    idx = np.arange(n)
    hit = idx == root
    cur = idx.copy()
    while (cur > 0).any():
        cur = np.where(cur > 0, (cur - 1) // 2, -1)
        hit |= cur == root
    return int(hit.sum())


@pytest.mark.parametrize("n", list(range(1, 70)) + [127, 128, 129, 255, 256, 257, 1000, 2047, 2048, 2049])
def test_left_size_matches_enumeration(n):
    assert oracle.left_size(n) == _subtree_size_by_ancestry(n, 1) if n > 1 else oracle.left_size(n) == 0


def test_parent_child_identities():
    n = np.arange(0, 1 << 20)
    parent = lambda c: (c + 1) // 2 - 1  # noqa: E731  (Sec. 3.2 parent rule)
    assert np.array_equal(parent(2 * n + 1), n)
    assert np.array_equal(parent(2 * n + 2), n)
    assert parent(np.array([0]))[0] == -1


# ---------------------------------------------------------------- builder

def test_six_point_tree():
    g = json.load(open(GOLDEN))
    pts = np.array(g["points"], dtype=np.float32)
    assert oracle.build(pts).tolist() == g["tree_ids"]


def _check_tree_property(pts: np.ndarray, node_pid: np.ndarray):
    """The level-order array is the unique complete tree whose every node
    separates its subtrees in its level's dimension (mod D) under the
    (coordinate, input index) order.  Checked bottom-up with subtree min/max
    keys, independently of how the tree was built."""
    N, D = pts.shape
    assert sorted(node_pid.tolist()) == list(range(N))
    # per node and dim: key = (coord, id); track subtree min and max keys
    coords = pts[node_pid].astype(np.float64)
    ids = node_pid.astype(np.int64)
    kmin_c = coords.copy()
    kmin_i = np.repeat(ids[:, None], D, axis=1)
    kmax_c = coords.copy()
    kmax_i = kmin_i.copy()

    def less(ac, ai, bc, bi):
        return (ac < bc) | ((ac == bc) & (ai < bi))

    for t in range(N - 1, -1, -1):
        for c in (2 * t + 1, 2 * t + 2):
            if c < N:
                m = less(kmin_c[c], kmin_i[c], kmin_c[t], kmin_i[t])
                kmin_c[t] = np.where(m, kmin_c[c], kmin_c[t])
                kmin_i[t] = np.where(m, kmin_i[c], kmin_i[t])
                m = less(kmax_c[t], kmax_i[t], kmax_c[c], kmax_i[c])
                kmax_c[t] = np.where(m, kmax_c[c], kmax_c[t])
                kmax_i[t] = np.where(m, kmax_i[c], kmax_i[t])
    for t in range(N):
        d = int(math.floor(math.log2(t + 1))) % D
        l, r = 2 * t + 1, 2 * t + 2
        if l < N:
            assert less(kmax_c[l, d], kmax_i[l, d], coords[t, d], ids[t]), t
        if r < N:
            assert less(coords[t, d], ids[t], kmin_c[r, d], kmin_i[r, d]), t


@pytest.mark.parametrize("N,D,seed", [(1, 3, 0), (2, 3, 1), (3, 2, 2), (7, 3, 3), (100, 3, 4),
                                      (257, 2, 5), (500, 4, 6), (333, 8, 7), (64, 1, 8), (1000, 3, 9)])
def test_build_separation_property(N, D, seed):
    g = np.random.default_rng(seed)
    pts = g.integers(0, 6, size=(N, D)).astype(np.float32)  # many ties
    if seed % 2:
        pts = g.random((N, D)).astype(np.float32)
    _check_tree_property(pts, oracle.build(pts))


def test_build_signed_zero_and_ties():
    pts = np.array([[0.0], [-0.0], [0.0], [-0.0], [1.0]], dtype=np.float32)
    node_pid = oracle.build(pts)
    _check_tree_property(pts, node_pid)
    # -0 == +0 under float <, so ties resolve by index: sorted order 0,1,2,3,4
    # L(5) = 3 -> root holds index 3
    assert node_pid[0] == 3


def test_build_rejects_nonfinite():
    pts = np.zeros((4, 3), dtype=np.float32)
    pts[2, 1] = np.nan
    with pytest.raises(ValueError):
        oracle.build(pts)


# ---------------------------------------------------------------- definition

def _numpy_knn(pts, qs, k, max_radius):
    """Independent statement of the result: d2 per term in float32 summed in
    coordinate order, filter d2 <= r2, lexsort by (d2, id), first k."""
    r2 = np.float32(max_radius) * np.float32(max_radius)
    Q = qs.shape[0]
    ids = np.full((Q, k), -1, dtype=np.int32)
    d2 = np.full((Q, k), np.inf, dtype=np.float32)
    for i in range(Q):
        diff = (pts - qs[i]).astype(np.float32)
        t = (diff * diff).astype(np.float32)
        s = t[:, 0].copy()
        for j in range(1, pts.shape[1]):
            s = (s + t[:, j]).astype(np.float32)
        cand = np.nonzero(s <= r2)[0]
        order = cand[np.lexsort((cand, s[cand]))][:k]
        ids[i, : len(order)] = order
        d2[i, : len(order)] = s[order]
    return ids, d2


@pytest.mark.parametrize("seed", range(6))
def test_brute_matches_numpy_definition(seed):
    g = np.random.default_rng(100 + seed)
    N, D = int(g.integers(1, 80)), int(g.integers(1, 9))
    pts = g.integers(0, 4, size=(N, D)).astype(np.float32) * np.float32(0.25)
    if seed % 2:
        pts = g.random((N, D)).astype(np.float32)
    qs = g.random((40, D)).astype(np.float32)
    for k in (1, 3, 8, N + 2):
        for r in (math.inf, 0.3, 0.0):
            a = oracle.knn_brute(pts, qs, k, r)
            b = _numpy_knn(pts, qs, k, r)
            assert np.array_equal(a[0], b[0])
            assert np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))


@pytest.mark.parametrize("threads", [1, 3, 7, 64])
def test_threaded_brute_equals_single_call(threads):
    """The threaded entry splits the queries into ragged ranges (and has more
    threads than queries at 64): the same bits as one call over all queries."""
    g = np.random.default_rng(41)
    pts = g.random((700, 3)).astype(np.float32)
    qs = g.random((50, 3)).astype(np.float32)
    for k, r in ((1, math.inf), (8, 0.1)):
        a = oracle.knn_brute(pts, qs, k, r)
        b = oracle.knn_brute_threaded(pts, qs, k, r, threads)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))


@pytest.mark.parametrize("threads", [2, 5, 16])
def test_parallel_builders_equal_serial(threads):
    """The threaded driver of the recursive builders (subtrees of the top
    levels in their own threads) gives the serial builders' trees: both split
    rules, ties on every dimension, ragged and complete sizes, sizes below the
    size at which subtrees stop spawning threads."""
    g = np.random.default_rng(threads)
    for N, D in ((1 << 15, 3), (50001, 3), (30000, 2), (9000, 5), (1000, 3)):
        pts = g.random((N, D)).astype(np.float32)
        pts[::5, 0] = 0.25
        pts[::7, D - 1] = np.float32(-0.0)
        pts[::11] = pts[3]
        assert np.array_equal(oracle.build(pts, threads=threads), oracle.build(pts))
        if D <= 3:
            a, b = oracle.build_widest(pts, threads=threads), oracle.build_widest(pts)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_threaded_traversal_equals_single_call(threads):
    """The threaded traversal (chunks of queries claimed by host threads) gives
    the single call's ids, distance bits and processed-node counts, for both
    split rules."""
    g = np.random.default_rng(43)
    pts = g.random((3000, 3)).astype(np.float32)
    qs = (g.random((777, 3)) * 1.4 - 0.2).astype(np.float32)
    pid = oracle.build(pts)
    wpid, wdims = oracle.build_widest(pts)
    for k, r in ((1, math.inf), (8, math.inf), (5, 0.05)):
        a = oracle.knn_tree(pts, pid, qs, k, r)
        b = oracle.knn_tree_threaded(pts, pid, qs, k, r, threads=threads)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))
        assert np.array_equal(a[2], b[2])
        c = oracle.knn_tree_dims(pts, wpid, wdims, qs, k, r)
        d = oracle.knn_tree_threaded(pts, wpid, qs, k, r, node_dim=wdims, threads=threads)
        assert np.array_equal(c[0], d[0]) and np.array_equal(c[1].view(np.uint32), d[1].view(np.uint32))
        assert np.array_equal(c[2], d[2])


def test_zero_radius_returns_exact_duplicates_only():
    g = np.random.default_rng(7)
    pts = g.integers(0, 3, size=(60, 2)).astype(np.float32)
    qs = pts[:10].copy()
    ids, d2 = oracle.knn_brute(pts, qs, 60, 0.0)
    for i in range(10):
        want = np.nonzero((pts == qs[i]).all(axis=1))[0]
        got = ids[i][ids[i] >= 0]
        assert got.tolist() == want.tolist()
        assert (d2[i][: len(want)] == 0).all()


def test_k_at_least_n_returns_all_sorted():
    g = np.random.default_rng(8)
    pts = g.random((17, 3)).astype(np.float32)
    q = g.random((1, 3)).astype(np.float32)
    ids, d2 = oracle.knn_brute(pts, q, 20, math.inf)
    assert sorted(ids[0, :17].tolist()) == list(range(17))
    assert ids[0, 17:].tolist() == [-1, -1, -1] and np.isinf(d2[0, 17:]).all()
    assert (np.diff(d2[0, :17]) >= 0).all()


def test_one_dimension_is_sorted_array_search():
    """D = 1: the nearest point is a neighbour of the insertion position in
    the sorted coordinates (textbook)."""
    g = np.random.default_rng(9)
    x = np.unique(g.random(500).astype(np.float32))
    pts = g.permutation(x)[:, None]
    qs = g.random((300, 1)).astype(np.float32)
    ids, d2 = oracle.knn_brute(pts, qs, 1)
    xs = np.sort(x)
    for i, q in enumerate(qs[:, 0]):
        j = np.searchsorted(xs, q)
        cands = [c for c in (j - 1, j) if 0 <= c < len(xs)]
        best = min(cands, key=lambda c: (np.float32(xs[c] - q) ** 2, c))
        assert pts[ids[i, 0], 0] == xs[best]


def test_fp64_brute_matches_lexicographic_selection_on_ties():
    """On small integer coordinates every squared distance is an exact integer
    in both precisions, so equal distances are common and the FP64 selection
    must be the k smallest (d2, index) pairs, as the FP32 one is."""
    g = np.random.default_rng(11)
    pts = g.integers(-3, 4, size=(300, 3)).astype(np.float32)
    qs = g.integers(-3, 4, size=(60, 3)).astype(np.float32)
    exact = ((pts[None, :, :].astype(np.int64) - qs[:, None, :].astype(np.int64)) ** 2).sum(axis=2)
    for k in (1, 7, 40, 301):
        i64, d64 = oracle.knn_brute_f64(pts, qs, k)
        for q in range(len(qs)):
            order = np.lexsort((np.arange(len(pts)), exact[q]))[:k]
            n = len(order)
            assert i64[q, :n].tolist() == order.tolist()
            assert d64[q, :n].tolist() == exact[q, order].astype(np.float64).tolist()
            assert (i64[q, n:] == -1).all() and np.isinf(d64[q, n:]).all()


def test_fp32_matches_fp64_up_to_rounding():
    g = np.random.default_rng(10)
    pts = g.random((3000, 3)).astype(np.float32)
    qs = g.random((200, 3)).astype(np.float32)
    k = 8
    i32, d32 = oracle.knn_brute(pts, qs, k)
    i64, d64 = oracle.knn_brute_f64(pts, qs, k)
    # each FP32 distance is within a few ulps of the exact one
    exact = np.array([[np.sum((pts[j].astype(np.float64) - qs[q].astype(np.float64)) ** 2) for j in i32[q]]
                      for q in range(len(qs))])
    assert np.allclose(d32, exact, rtol=4 * 2.0 ** -23, atol=0)
    # the k-th FP32 distance equals the exact k-th up to rounding; ids agree
    # except where two exact distances fall within rounding of each other
    assert np.allclose(d32[:, -1], d64[:, -1], rtol=8 * 2.0 ** -23)
    agree = (i32 == i64).mean()
    assert agree > 0.99


# ---------------------------------------------------------------- traversal

def test_six_point_traces():
    g = json.load(open(GOLDEN))
    pts = np.array(g["points"], dtype=np.float32)
    node_pid = np.array(g["tree_ids"], dtype=np.int32)
    for tr in g["traces"]:
        for fn in (oracle.knn_recursive, oracle.knn_stackfree):
            ids, d2, visits, _ = fn(pts, node_pid, tr["query"], tr["k"], math.inf, tr["ordered"])
            assert ids.tolist() == tr["ids"], (fn, tr)
            assert d2.tolist() == tr["d2"], (fn, tr)
            assert visits.tolist() == tr["visits"], (fn, tr)


def _cases():
    for seed in range(12):
        g = np.random.default_rng(200 + seed)
        N = int(g.integers(1, 70))
        D = int(g.integers(1, 5))
        if seed % 3 == 0:
            pts = g.integers(0, 3, size=(N, D)).astype(np.float32)  # duplicates
        elif seed % 3 == 1:
            pts = np.repeat(g.random((N, 1)), D, axis=1).astype(np.float32)  # collinear
        else:
            pts = g.random((N, D)).astype(np.float32)
        qs = (g.random((25, D)) * 1.4 - 0.2).astype(np.float32)
        yield seed, pts, qs
    # integer grids: queries on the splitting planes (sd == 0, where the close
    # side is the left child), and many equal distances
    for seed in range(12, 16):
        g = np.random.default_rng(200 + seed)
        N = int(g.integers(2, 90))
        D = int(g.integers(1, 4))
        pts = g.integers(0, 3, size=(N, D)).astype(np.float32)
        qs = g.integers(-1, 4, size=(25, D)).astype(np.float32)
        yield seed, pts, qs


@pytest.mark.parametrize("seed,pts,qs", list(_cases()))
def test_traversals_match_brute_and_each_other(seed, pts, qs):
    node_pid = oracle.build(pts)
    N = len(pts)
    for k in (1, 2, 5, N + 1):
        for r in (math.inf, 0.35, 0.0):
            want_i, want_d = oracle.knn_brute(pts, qs, k, r)
            for q in range(len(qs)):
                runs = {}
                for ordered in (True, False):
                    for name, fn in (("rec", oracle.knn_recursive), ("sm", oracle.knn_stackfree)):
                        ids, d2, visits, steps = fn(pts, node_pid, qs[q], k, r, ordered)
                        assert ids.tolist() == want_i[q].tolist()
                        assert np.array_equal(d2.view(np.uint32), want_d[q].view(np.uint32))
                        runs[(ordered, name)] = (visits, steps)
                    # Sec. 3.1: same nodes, same order, as the recursion
                    assert np.array_equal(runs[(ordered, "rec")][0], runs[(ordered, "sm")][0])
                    assert np.array_equal(runs[(ordered, "rec")][1], runs[(ordered, "sm")][1])


def _preorder(N):
    out, stack = [], [0]
    while stack:
        n = stack.pop()
        if n < N:
            out.append(n)
            stack.extend([2 * n + 2, 2 * n + 1])
    return out


@pytest.mark.parametrize("N", [1, 2, 3, 6, 31, 32, 33, 100])
def test_unordered_unbounded_visits_every_node_once_in_preorder(N):
    g = np.random.default_rng(N)
    pts = g.random((N, 3)).astype(np.float32)
    node_pid = oracle.build(pts)
    q = g.random(3).astype(np.float32)
    _, _, visits, steps = oracle.knn_stackfree(pts, node_pid, q, N, math.inf, ordered=False)
    assert visits.tolist() == _preorder(N)
    # each valid node is stepped on at most three times, each missing child once
    counts = np.bincount(steps[steps < N], minlength=N)
    assert counts.max() <= 3


@pytest.mark.parametrize("seed", range(4))
def test_state_machine_steps_follow_the_three_cases(seed):
    """Sec. 3.2: a valid node is reached first from its parent (processed,
    then the close child), second from its close child (then the far child if
    in range, else the parent), third from its far child (then the parent); a
    missing node is left for its parent at once.  So in the step log every
    processed node occurs two or three times, first after its parent, and
    every other occurrence follows one of its children."""
    g = np.random.default_rng(600 + seed)
    N, D = int(g.integers(20, 300)), int(g.integers(1, 4))
    pts = g.random((N, D)).astype(np.float32)
    pid = oracle.build(pts)
    for q in g.random((10, D)).astype(np.float32):
        for k, r in ((1, math.inf), (5, math.inf), (3, 0.2)):
            _, _, visits, steps = oracle.knn_stackfree(pts, pid, q, k, r)
            steps = steps.tolist()
            assert steps[0] == 0 and steps[-1] == 0
            seen = {}
            for i, n in enumerate(steps):
                seen.setdefault(n, []).append(i)
            for n, at in seen.items():
                if n >= N:
                    # stepped into and straight back out to the parent
                    assert all(steps[i - 1] == (n - 1) // 2 and steps[i + 1] == (n - 1) // 2 for i in at)
                    continue
                assert len(at) in (2, 3), (n, at)
                assert at[0] == 0 if n == 0 else steps[at[0] - 1] == (n - 1) // 2
                for i in at[1:]:
                    assert steps[i - 1] in (2 * n + 1, 2 * n + 2)
                if len(at) == 3:
                    # the second and third arrivals come from different children
                    assert steps[at[1] - 1] != steps[at[2] - 1]
            # processed nodes are exactly the valid nodes reached, in first-arrival order
            assert visits.tolist() == [n for n in dict.fromkeys(steps) if n < N]


def test_ordered_visit_counts_uniform_3d():
    """Batch entry agrees with per-query entry; visit counts are positive and
    the ordered traversal processes far fewer nodes than there are points."""
    pts, qs = synth.uniform_small(4096, 256)
    node_pid = oracle.build(pts)
    ids, d2, nv = oracle.knn_tree(pts, node_pid, qs, 8)
    bi, bd = oracle.knn_brute(pts, qs, 8)
    assert np.array_equal(ids, bi) and np.array_equal(d2, bd)
    for q in (0, 17, 255):
        _, _, visits, _ = oracle.knn_stackfree(pts, node_pid, qs[q], 8)
        assert len(visits) == nv[q]
    assert 8 <= nv.min() and nv.mean() < 0.1 * len(pts)


def test_descent_leaf_is_first_leaf_of_ordered_traversal():
    """The greedy close-child descent ends where the ordered traversal first
    turns back: the last node stepped on before the first missing child."""
    pts, qs = synth.uniform_small(1000, 50)
    node_pid = oracle.build(pts)
    N = len(pts)
    leaf_d2 = oracle.descent_leaf_d2(pts, node_pid, qs)
    for i in range(len(qs)):
        _, _, _, steps = oracle.knn_stackfree(pts, node_pid, qs[i], 1)
        first_missing = int(np.argmax(steps >= N))
        leaf = steps[first_missing - 1]
        diff = (pts[node_pid[leaf]] - qs[i]).astype(np.float32)
        t = (diff * diff).astype(np.float32)
        assert leaf_d2[i] == np.float32(np.float32(t[0] + t[1]) + t[2])


@pytest.mark.parametrize("widest", [False, True])
@pytest.mark.parametrize("N", [2, 3, 10, 255, 256, 1000])
def test_descent_from_a_leaf_point_ends_on_it(N, widest):
    """With distinct coordinates every split separates strictly, so a query
    equal to the point stored at a leaf follows the close child down to that
    leaf (the last node N - 1 included) and finds distance 0; on a tree with
    the split dimension stored per node only if the descent reads each node's
    own dimension (the points are stretched along x, so the stored dimensions
    differ from level mod D)."""
    g = np.random.default_rng(N)
    pts = (g.random((N, 3)) * np.array([8.0, 1.0, 0.25])).astype(np.float32)
    dims = None
    if widest:
        pid, dims = oracle.build_widest(pts)
        if N >= 255:
            assert (dims != np.array([oracle_level(n) % 3 for n in range(N)])).mean() > 0.3
    else:
        pid = oracle.build(pts)
    leaves = [n for n in range(N) if 2 * n + 1 >= N]
    assert N - 1 in leaves
    d2 = oracle.descent_leaf_d2(pts, pid, pts[pid[leaves]], node_dim=dims)
    assert (d2 == 0).all()


def oracle_level(n: int) -> int:
    return (n + 1).bit_length() - 1


def test_descent_leaf_with_stored_dims_bounds_the_nearest():
    """The descent ends on a point of the set, so its distance is at least the
    brute-force nearest distance and equals it for queries at stored points;
    with the level-mod-D dimensions passed explicitly it is the plain descent."""
    pts, qs = synth.uniform_small(2000, 300)
    pid, dims = oracle.build_widest(pts)
    d2 = oracle.descent_leaf_d2(pts, pid, qs, node_dim=dims)
    _, bd = oracle.knn_brute(pts, qs, 1)
    assert (d2 >= bd[:, 0]).all() and (d2 > bd[:, 0]).any()
    plain = oracle.build(pts)
    lvl = np.array([oracle_level(n) % 3 for n in range(len(pts))], dtype=np.uint8)
    assert np.array_equal(oracle.descent_leaf_d2(pts, plain, qs, node_dim=lvl).view(np.uint32),
                          oracle.descent_leaf_d2(pts, plain, qs).view(np.uint32))


# ---------------------------------------------------------------- MLP

def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(11)
    xs = np.concatenate([g.standard_normal(2000) * 10.0 ** g.integers(-8, 8, 2000),
                         [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e38]]).astype(np.float32)
    want = torch.from_numpy(xs).to(torch.bfloat16).to(torch.float32).numpy()
    got = np.array([oracle.round_bf16(float(x)) for x in xs], dtype=np.float32)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def _numpy_mlp(params, H, x):
    W1 = params[: 4 * H].reshape(H, 4)
    b1 = params[4 * H: 5 * H]
    W2 = params[5 * H: 5 * H + H * H].reshape(H, H)
    b2 = params[5 * H + H * H: 6 * H + H * H]
    w3 = params[6 * H + H * H: 7 * H + H * H]
    b3 = params[7 * H + H * H]
    h1 = np.maximum(x @ W1.T + b1, 0)
    h2 = np.maximum(h1 @ W2.T + b2, 0)
    return h2 @ w3 + b3


def test_mlp_forward_matches_matrix_form():
    H = 16
    g = np.random.default_rng(12)
    p = g.standard_normal(oracle.mlp_param_count(H)) * 0.5
    x = g.standard_normal((64, 4))
    assert np.allclose(oracle.mlp_forward(p, H, x), _numpy_mlp(p, H, x), rtol=1e-12, atol=1e-12)


def test_mlp_gradient_matches_finite_differences():
    H = 8
    g = np.random.default_rng(13)
    p = g.standard_normal(oracle.mlp_param_count(H)) * 0.5
    x = g.standard_normal((32, 4))
    lab = g.standard_normal(32)
    loss, grad = oracle.mlp_loss_grad(p, H, x, lab)
    assert math.isclose(loss, float(np.mean((_numpy_mlp(p, H, x) - lab) ** 2)), rel_tol=1e-12)
    eps = 1e-6
    for i in range(len(p)):
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (np.mean((_numpy_mlp(pp, H, x) - lab) ** 2) - np.mean((_numpy_mlp(pm, H, x) - lab) ** 2)) / (2 * eps)
        assert abs(fd - grad[i]) <= 1e-5 * max(1.0, abs(fd)), i


def _bf16(v):
    """Round float32 values to the nearest bfloat16 (ties to even) through torch."""
    import torch

    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).to(torch.bfloat16).float().numpy()


def _bf16_params(H, seed, scale=0.5):
    g = np.random.default_rng(seed)
    p = (g.standard_normal(oracle.mlp_param_count(H)) * scale).astype(np.float32)
    return _bf16(p).astype(np.float64)


def _simulate_bf16_in(p, H, x, order):
    """An FP32 evaluation with the hidden activations rounded to bfloat16:
    layer 1 unfused (products rounded) or through FP64 then rounded once
    (a fused chain's accuracy), sums left to right or reversed."""
    f = np.float32
    W1 = p[: 4 * H].reshape(H, 4).astype(f)
    b1 = p[4 * H: 5 * H].astype(f)
    W2 = p[5 * H: 5 * H + H * H].reshape(H, H).astype(f)
    b2 = p[5 * H + H * H: 6 * H + H * H].astype(f)
    w3 = p[6 * H + H * H: 7 * H + H * H].astype(f)
    b3 = f(p[-1])
    xs = x.astype(f)
    if order == "fused":
        z1 = (b1.astype(np.float64) + xs.astype(np.float64) @ W1.T.astype(np.float64)).astype(f)
    else:
        z1 = np.repeat(b1[None, :], xs.shape[0], 0)
        for j in range(4):
            z1 = (z1 + (W1[:, j][None, :] * xs[:, j:j + 1]).astype(f)).astype(f)
    h1 = _bf16(np.maximum(z1, f(0)))
    idx = range(H) if order != "reversed" else range(H - 1, -1, -1)
    acc = np.zeros((xs.shape[0], H), dtype=f)
    for i in idx:
        acc = (acc + (h1[:, i:i + 1] * W2[:, i][None, :]).astype(f)).astype(f)
    h2 = np.maximum((acc + b2[None, :]).astype(f), f(0))
    y = np.full(xs.shape[0], b3, dtype=f)
    for j in idx:
        y = (y + (w3[j] * h2[:, j]).astype(f)).astype(f)
    return y.astype(np.float64)


def test_mlp_forward_bound_value_is_the_fp64_forward():
    H = 16
    p = _bf16_params(H, 15)
    x = np.random.default_rng(16).standard_normal((200, 4)).astype(np.float32).astype(np.float64)
    y, bound = oracle.mlp_forward_bound(p, H, x)
    assert np.array_equal(y.view(np.uint64), oracle.mlp_forward(p, H, x).view(np.uint64))
    assert np.all(bound > 0)


@pytest.mark.parametrize("order", ["unfused", "fused", "reversed"])
def test_mlp_forward_bound_covers_bf16_in_fp32_evaluations(order):
    """Simulated BF16-in / FP32 evaluations in three orders stay within the
    per-sample bound, on the model's width and on a narrow one."""
    for H, seed in ((64, 17), (8, 18)):
        p = _bf16_params(H, seed)
        x = np.random.default_rng(seed + 100).standard_normal((3000, 4)).astype(np.float32).astype(np.float64)
        y, bound = oracle.mlp_forward_bound(p, H, x)
        sim = _simulate_bf16_in(p, H, x, order)
        assert np.all(np.abs(sim - y) <= bound), float(np.max(np.abs(sim - y) / bound))
        # and the rounding does show: the bound is not vacuous for these models
        assert np.max(np.abs(sim - y)) > 0


def test_mlp_forward_bound_is_tight_for_one_rounded_activation():
    """A hidden activation of 1 + 2^-8 lies halfway between the bfloat16
    neighbours 1 and 1 + 2^-7 and rounds to 1 (ties to even): the model's
    output 1 + 2^-8 becomes 1, an error of 2^-8.  The bound must cover it, and
    by little (the FP32 terms add only about 2^-20)."""
    H = 1
    p = np.zeros(oracle.mlp_param_count(H))
    p[0] = 1.0            # W1[0][0]
    p[4] = 2.0 ** -8      # b1
    p[5] = 1.0            # W2
    p[7] = 1.0            # w3
    x = np.array([[1.0, 0, 0, 0]])
    y, bound = oracle.mlp_forward_bound(p, H, x)
    assert y[0] == 1.0 + 2.0 ** -8
    assert _simulate_bf16_in(p, H, x, "unfused")[0] == 1.0
    assert 2.0 ** -8 <= bound[0] <= 1.01 * 2.0 ** -8


def test_mlp_forward_bound_covers_cancellation_in_layer1():
    """Layer 1 with cancelling terms: (1 + 2^-7)(1 + 2^-20) is 1 + 2^-7 + 2^-20
    + 2^-27 exactly and 1 + 2^-7 + 2^-20 in FP32, so with the second term
    -(1 + 2^-7 + 2^-20) an FP32 evaluation gets 0 where the model has 2^-27.
    Only the bound's FP32 allowance of layer 1 covers that (the activation is
    far below the bfloat16 level)."""
    H = 1
    p = np.zeros(oracle.mlp_param_count(H))
    p[0] = 1.0 + 2.0 ** -7     # W1[0][0]
    p[1] = -1.0                # W1[0][1]
    p[5] = 1.0                 # W2
    p[7] = 1.0                 # w3
    x = np.array([[1.0 + 2.0 ** -20, 1.0 + 2.0 ** -7 + 2.0 ** -20, 0, 0]])
    y, bound = oracle.mlp_forward_bound(p, H, x)
    assert y[0] == 2.0 ** -27
    assert _simulate_bf16_in(p, H, x, "unfused")[0] == 0.0
    assert bound[0] >= 2.0 ** -27


def _simulate_bf16_in_grad(p, H, x, lab, reverse=False):
    """An FP32 training step with BF16 operands in the 64 x 64 contractions:
    the hidden activations of layer 1 and the gradient at the hidden layer's
    pre-activations rounded to bfloat16 there, sums over samples and units in
    FP32 (in index order, or reversed).  Returns (loss, grad float64[P])."""
    f = np.float32
    W1 = p[: 4 * H].reshape(H, 4).astype(f)
    b1 = p[4 * H: 5 * H].astype(f)
    W2 = p[5 * H: 5 * H + H * H].reshape(H, H).astype(f)
    b2 = p[5 * H + H * H: 6 * H + H * H].astype(f)
    w3 = p[6 * H + H * H: 7 * H + H * H].astype(f)
    b3 = f(p[-1])
    xs, ls = x.astype(f), lab.astype(f)
    n = xs.shape[0]
    order = range(n - 1, -1, -1) if reverse else range(n)
    units = range(H - 1, -1, -1) if reverse else range(H)
    z1 = np.repeat(b1[None, :], n, 0)
    for m in range(4):
        z1 = (z1 + (W1[:, m][None, :] * xs[:, m:m + 1]).astype(f)).astype(f)
    h1b = _bf16(np.maximum(z1, f(0)))
    z2 = np.zeros((n, H), dtype=f)
    for j in units:
        z2 = (z2 + (h1b[:, j:j + 1] * W2[:, j][None, :]).astype(f)).astype(f)
    z2 = (z2 + b2[None, :]).astype(f)
    h2 = np.maximum(z2, f(0))
    y = np.full(n, b3, dtype=f)
    for i in units:
        y = (y + (w3[i] * h2[:, i]).astype(f)).astype(f)
    err = (y - ls).astype(f)
    go = ((f(2) * err).astype(f) * f(1.0 / n)).astype(f)
    g2 = np.where(z2 > 0, (go[:, None] * w3[None, :]).astype(f), f(0)).astype(f)
    g2b = _bf16(g2)
    dH1 = np.zeros((n, H), dtype=f)
    for i in units:
        dH1 = (dH1 + (g2b[:, i:i + 1] * W2[i, :][None, :]).astype(f)).astype(f)
    g1 = np.where(z1 > 0, dH1, f(0)).astype(f)
    gW1 = np.zeros((H, 4), f); gb1 = np.zeros(H, f); gW2 = np.zeros((H, H), f)
    gb2 = np.zeros(H, f); gw3 = np.zeros(H, f); gb3 = f(0); loss = f(0)
    for s_ in order:
        gW1 = (gW1 + (g1[s_][:, None] * xs[s_][None, :]).astype(f)).astype(f)
        gb1 = (gb1 + g1[s_]).astype(f)
        gW2 = (gW2 + (g2b[s_][:, None] * h1b[s_][None, :]).astype(f)).astype(f)
        gb2 = (gb2 + g2[s_]).astype(f)
        gw3 = (gw3 + (go[s_] * h2[s_]).astype(f)).astype(f)
        gb3 = f(gb3 + go[s_])
        loss = f(loss + f(err[s_] * err[s_]))
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]]).astype(np.float64)
    return float(loss) / n, grad


@pytest.mark.parametrize("reverse", [False, True])
def test_mlp_grad_bound_covers_bf16_in_fp32_training(reverse):
    """Simulated BF16-in / FP32 training steps stay within the per-parameter
    bound (and the loss within its bound), on the model's width and a narrow
    one; the rounding does show in the simulated gradient."""
    for H, seed, n in ((64, 31, 700), (8, 32, 300)):
        p = _bf16_params(H, seed, 0.4)
        g = np.random.default_rng(seed + 7)
        x = g.standard_normal((n, 4)).astype(np.float32).astype(np.float64)
        lab = g.standard_normal(n).astype(np.float32).astype(np.float64)
        loss, grad, bound, lbound = oracle.mlp_loss_grad_bound(p, H, x, lab)
        l2, g2 = oracle.mlp_loss_grad(p, H, x, lab)
        assert loss == l2 and np.array_equal(grad, g2)
        sl, sg = _simulate_bf16_in_grad(p, H, x, lab, reverse)
        assert np.all(np.abs(sg - grad) <= bound), float(np.max(np.abs(sg - grad) / np.maximum(bound, 1e-300)))
        assert abs(sl - loss) <= lbound
        assert np.max(np.abs(sg - grad)) > 0


def test_mlp_grad_bound_tight_for_one_rounded_activation():
    """One sample, one hidden unit of activation 1 + 2^-8 (rounds to 1 in
    bfloat16), identity weights, label 0: the model's dW2 is
    2 (1 + 2^-8)^2, the BF16-in step's 2; the bound covers the difference
    and is within a factor of three of it."""
    H = 1
    p = np.zeros(oracle.mlp_param_count(H))
    p[0] = 1.0            # W1[0][0]
    p[4] = 2.0 ** -8      # b1
    p[5] = 1.0            # W2
    p[7] = 1.0            # w3
    x = np.array([[1.0, 0, 0, 0]])
    lab = np.array([0.0])
    loss, grad, bound, _ = oracle.mlp_loss_grad_bound(p, H, x, lab)
    _, sg = _simulate_bf16_in_grad(p, H, x, lab)
    assert grad[5] == 2.0 * (1.0 + 2.0 ** -8) ** 2 and sg[5] == 2.0
    d = grad[5] - sg[5]
    assert d <= bound[5] <= 3.0 * d


def test_mlp_grad_bound_covers_rounded_back_propagation():
    """h1 = 1 exactly, label -(4 + 2^-6): the error 5 + 2^-6 gives go =
    10 + 2^-5, which lies halfway between the bfloat16 neighbours 10 and
    10.0625 and rounds to 10.  The gradient at the first layer's bias is that
    operand times W2 = 1: 10 instead of 10 + 2^-5; only the bound's rounding
    allowance for the back-propagated operand covers it."""
    H = 1
    p = np.zeros(oracle.mlp_param_count(H))
    p[0] = 1.0    # W1[0][0]
    p[5] = 1.0    # W2
    p[7] = 1.0    # w3
    x = np.array([[1.0, 0, 0, 0]])
    lab = np.array([-(4.0 + 2.0 ** -6)])
    loss, grad, bound, _ = oracle.mlp_loss_grad_bound(p, H, x, lab)
    _, sg = _simulate_bf16_in_grad(p, H, x, lab)
    assert grad[4] == 10.0 + 2.0 ** -5 and sg[4] == 10.0
    assert np.all(np.abs(sg - grad) <= bound)


def test_mlp_grad_bound_covers_rounded_activation_in_dw2():
    """An activation of 1 + 2^-8 (rounds to 1) with label -(1 + 2^-8): the
    weight gradient dW2 = go h1 is (4 + 2^-6)(1 + 2^-8) for the model and 4
    for the rounded step; the bound must carry the activation's error into
    the weight gradient."""
    H = 1
    p = np.zeros(oracle.mlp_param_count(H))
    p[0] = 1.0            # W1[0][0]
    p[4] = 2.0 ** -8      # b1
    p[5] = 1.0            # W2
    p[7] = 1.0            # w3
    x = np.array([[1.0, 0, 0, 0]])
    lab = np.array([-(1.0 + 2.0 ** -8)])
    loss, grad, bound, _ = oracle.mlp_loss_grad_bound(p, H, x, lab)
    _, sg = _simulate_bf16_in_grad(p, H, x, lab)
    assert sg[5] == 4.0 and grad[5] > 4.0 + 2.0 ** -6
    assert np.all(np.abs(sg - grad) <= bound)


def test_mlp_grad_bound_admits_a_flipped_mask():
    """A hidden pre-activation of 2^-12 is within its forward bound of 0: the
    layer-1 activation 1 + 2^-9 rounds to 1 in bfloat16, so with the bias
    -(1 + 2^-9) + 2^-12 the model's pre-activation is 2^-12 and the rounded
    evaluation's is 2^-12 - 2^-9 < 0.  Its ReLU switches off there and the
    unit's gradient is 0 instead of go w3; the bound admits both values."""
    H = 1
    p = np.zeros(oracle.mlp_param_count(H))
    p[0] = 1.0                    # W1[0][0]
    p[4] = 2.0 ** -9              # b1: h1 = 1 + 2^-9, rounds to 1
    p[5] = 1.0                    # W2
    p[6] = -(1.0 + 2.0 ** -9) + 2.0 ** -12   # b2: z2 = 2^-12 exactly, 2^-12 - 2^-9 < 0 after rounding
    p[7] = 1.0                    # w3
    x = np.array([[1.0, 0, 0, 0]])
    lab = np.array([-1.0])
    loss, grad, bound, _ = oracle.mlp_loss_grad_bound(p, H, x, lab)
    _, sg = _simulate_bf16_in_grad(p, H, x, lab)
    assert grad[6] != 0.0 and sg[6] == 0.0          # db2: the mask switched off
    assert np.all(np.abs(sg - grad) <= bound)


def test_mlp_forward_bound_value_exact_for_integer_model():
    """Small-integer weights, biases and inputs: every value is exact in
    bfloat16 and FP32, so a BF16-in / FP32 evaluation gives the FP64 forward's
    value exactly (a dropped bias or a transposed matrix would show here)."""
    H = 16
    g = np.random.default_rng(14)
    p = np.zeros(oracle.mlp_param_count(H))
    p[: 4 * H] = g.integers(-2, 3, 4 * H)
    p[4 * H: 5 * H] = g.integers(-3, 4, H)
    p[5 * H: 5 * H + H * H] = g.integers(-1, 2, H * H)
    p[5 * H + H * H:] = g.integers(-2, 3, len(p) - 5 * H - H * H)
    x = g.integers(-4, 5, size=(50, 4)).astype(np.float64)
    y, bound = oracle.mlp_forward_bound(p, H, x)
    assert np.array_equal(_simulate_bf16_in(p, H, x, "unfused"), y)
    assert np.all(bound >= 0)


# ---------------------------------------------------------------- stored split dimension

def _check_widest_tree(pts, node_pid, node_dim):
    """Every node's stored dimension is the widest extent (max - min in float32,
    ties to the lowest index) of its subtree's points, and the node separates
    its subtrees in that dimension under the (coordinate, index) order."""
    N, D = pts.shape
    assert sorted(node_pid.tolist()) == list(range(N))
    c = pts[node_pid]
    lo, hi = c.copy(), c.copy()
    ids = node_pid.astype(np.int64)
    kmin = [((c[:, d].astype(np.float64)), ids.copy()) for d in range(D)]
    for t in range(N - 1, -1, -1):
        for ch in (2 * t + 1, 2 * t + 2):
            if ch < N:
                lo[t] = np.minimum(lo[t], lo[ch])
                hi[t] = np.maximum(hi[t], hi[ch])
    ext = (hi - lo).astype(np.float32)
    assert np.array_equal(node_dim, np.argmax(ext, axis=1).astype(np.uint8))

    def keys(t, d):
        # all (coord, id) keys of subtree t in dimension d
        out, stack = [], [t]
        while stack:
            u = stack.pop()
            if u < N:
                out.append((float(c[u, d]), int(ids[u])))
                stack += [2 * u + 1, 2 * u + 2]
        return out

    for t in range(N):
        d = int(node_dim[t])
        me = (float(c[t, d]), int(ids[t]))
        if 2 * t + 1 < N:
            assert max(keys(2 * t + 1, d)) < me, t
        if 2 * t + 2 < N:
            assert me < min(keys(2 * t + 2, d)), t


def test_widest_six_point_example():
    g = json.load(open(GOLDEN))
    pts = np.array(g["points"], dtype=np.float32)
    node_pid, node_dim = oracle.build_widest(pts)
    # root: x extent 7 > y extent 6; (5,4)'s points: y 4 > x 3; (9,6)'s: y 5 > x 1;
    # single points have extent 0 everywhere -> dimension 0
    assert node_dim.tolist() == [0, 1, 1, 0, 0, 0]
    assert node_pid.tolist() == g["tree_ids"]


@pytest.mark.parametrize("N,D,seed", [(1, 3, 0), (2, 2, 1), (9, 3, 2), (130, 3, 3), (300, 2, 4), (257, 1, 5)])
def test_widest_builder_property(N, D, seed):
    g = np.random.default_rng(seed)
    pts = (g.random((N, D)) * np.array([1.0, 3.0, 0.5][:D])).astype(np.float32)
    if seed % 2:
        pts = g.integers(0, 5, size=(N, D)).astype(np.float32)  # ties in extents and coordinates
    node_pid, node_dim = oracle.build_widest(pts)
    _check_widest_tree(pts, node_pid, node_dim)


@pytest.mark.parametrize("seed", range(4))
def test_widest_traversal_matches_brute(seed):
    g = np.random.default_rng(300 + seed)
    N, D = int(g.integers(1, 300)), int(g.integers(1, 4))
    pts = (g.random((N, D)) * g.uniform(0.1, 3.0, D)).astype(np.float32)
    if seed % 2:
        pts = g.integers(0, 4, size=(N, D)).astype(np.float32)
    qs = (g.random((60, D)) * 1.2 - 0.1).astype(np.float32)
    node_pid, node_dim = oracle.build_widest(pts)
    for k, r in ((1, math.inf), (8, math.inf), (5, 0.3)):
        want = oracle.knn_brute(pts, qs, k, r)
        for ordered in (True, False):
            got = oracle.knn_tree_dims(pts, node_pid, node_dim, qs, k, r, ordered)
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


# ---------------------------------------------------------------- range queries

@pytest.mark.parametrize("seed", range(3))
def test_radius_brute_equals_unbounded_knn_within_radius(seed):
    """The ball query is the kNN definition with k >= N and the same radius."""
    g = np.random.default_rng(400 + seed)
    N, D = 150, int(g.integers(1, 4))
    pts = g.integers(0, 5, size=(N, D)).astype(np.float32) * np.float32(0.25) if seed % 2 else \
        g.random((N, D)).astype(np.float32)
    qs = g.random((30, D)).astype(np.float32)
    r = 0.4
    counts, offsets, ids, d2 = oracle.radius_brute(pts, qs, r)
    ki, kd = oracle.knn_brute(pts, qs, N, r)
    for q in range(len(qs)):
        got = ids[offsets[q]:offsets[q + 1]]
        want = ki[q][ki[q] >= 0]
        assert counts[q] == len(want)
        assert sorted(got.tolist()) == sorted(want.tolist())
        order = np.argsort(got)
        assert np.array_equal(d2[offsets[q]:offsets[q + 1]][order].view(np.uint32),
                              kd[q][: len(want)][np.argsort(want)].view(np.uint32))


def test_box_brute_equals_mask():
    g = np.random.default_rng(7)
    pts = g.integers(0, 6, size=(300, 3)).astype(np.float32)
    lo = g.integers(0, 4, size=(40, 3)).astype(np.float32)
    hi = lo + g.integers(0, 3, size=(40, 3)).astype(np.float32)
    counts, offsets, ids = oracle.box_brute(pts, lo, hi)
    for q in range(40):
        want = np.nonzero(((pts >= lo[q]) & (pts <= hi[q])).all(axis=1))[0]
        assert ids[offsets[q]:offsets[q + 1]].tolist() == want.tolist()


# ------------------------------------------------- range queries on the tree

def _preorder_rank(N):
    """Preorder position of every node of a level-order complete tree (explicit stack)."""
    rank = np.empty(N, dtype=np.int64)
    stack, r = [0], 0
    while stack:
        n = stack.pop()
        if n >= N:
            continue
        rank[n] = r
        r += 1
        stack.append(2 * n + 2)
        stack.append(2 * n + 1)
    return rank


@pytest.mark.parametrize("seed", range(6))
def test_range_traversal_hits_equal_brute_in_preorder(seed):
    """The stack-free range traversal finds exactly the brute-force hit set, and
    (left child first, node before its subtrees) lists them in preorder."""
    g = np.random.default_rng(500 + seed)
    N, D = int(g.integers(1, 400)), int(g.integers(1, 5))
    pts = g.random((N, D)).astype(np.float32)
    if seed % 2:
        pts = g.integers(0, 5, size=(N, D)).astype(np.float32) * np.float32(0.25)
    widest = seed % 3 == 2 and D <= 3
    if widest:
        pid, dims = oracle.build_widest(pts)
    else:
        pid, dims = oracle.build(pts), None
    node_of = np.empty(N, dtype=np.int64)
    node_of[pid] = np.arange(N)
    rank = _preorder_rank(N)
    qs = (g.random((40, D)) * 1.2 - 0.1).astype(np.float32)
    qs[:10] = pts[g.integers(0, N, 10)]
    for r in (0.0, 0.1, 0.35, np.inf):
        c, off, ids, d2 = oracle.range_tree(pts, pid, qs, radius=r, node_dim=dims)
        wc, woff, wids, wd2 = oracle.radius_brute(pts, qs, r)
        assert np.array_equal(c, wc)
        for q in range(len(qs)):
            got, gd = ids[off[q]:off[q + 1]], d2[off[q]:off[q + 1]]
            o = np.argsort(got)
            assert np.array_equal(got[o], wids[woff[q]:woff[q + 1]])
            assert np.array_equal(gd[o].view(np.uint32), wd2[woff[q]:woff[q + 1]].view(np.uint32))
            assert np.all(np.diff(rank[node_of[got]]) > 0)
    lo = (g.random((40, D)) * 0.8).astype(np.float32)
    hi = lo + (g.random((40, D)) * 0.5).astype(np.float32)
    lo[:5], hi[:5] = pts[:5], pts[:5]
    c, off, ids, _ = oracle.range_tree(pts, pid, lo, hi, node_dim=dims)
    wc, woff, wids = oracle.box_brute(pts, lo, hi)
    assert np.array_equal(c, wc)
    for q in range(len(lo)):
        got = ids[off[q]:off[q + 1]]
        assert np.array_equal(np.sort(got), wids[woff[q]:woff[q + 1]])
        assert np.all(np.diff(rank[node_of[got]]) > 0)


def test_range_traversal_six_point_example():
    """Figure 1's six points: a ball of radius 3 around (7,2) holds (7,2) (d2 0),
    (5,4) (d2 8) and (8,1) (d2 2), not (9,6) (d2 20); the traversal meets them as
    the root, then in the left subtree, then in the right subtree."""
    gd = json.load(open(GOLDEN))
    pts = np.array(gd["points"], dtype=np.float32)
    pid = oracle.build(pts)
    q = np.array([[7.0, 2.0]], dtype=np.float32)
    c, off, ids, d2 = oracle.range_tree(pts, pid, q, radius=3.0)
    names = [tuple(pts[i].tolist()) for i in ids]
    assert names == [(7.0, 2.0), (5.0, 4.0), (8.0, 1.0)]
    assert d2.tolist() == [0.0, 8.0, 2.0]


def test_payload_reductions_integer_payload_exact():
    """Small-integer payloads sum exactly in FP32: the reductions equal integer
    sums over the brute-force hit sets; the density times pi R^2 gives the sum back."""
    g = np.random.default_rng(9)
    N, D, C = 3000, 3, 4
    pts = g.random((N, D)).astype(np.float32)
    pay = g.integers(-50, 50, size=(N, C)).astype(np.float32)
    pid = oracle.build(pts)
    qs = g.random((60, D)).astype(np.float32)
    r = 0.12
    _, woff, wids, _ = oracle.radius_brute(pts, qs, r)
    s, cnt = oracle.range_reduce(pts, pid, qs, r, pay, oracle.REDUCE_SUM)
    m, _ = oracle.range_reduce(pts, pid, qs, r, pay, oracle.REDUCE_MEAN)
    dn, _ = oracle.range_reduce(pts, pid, qs, r, pay, oracle.REDUCE_DENSITY)
    r2 = float(np.float32(r) * np.float32(r))
    for q in range(len(qs)):
        hit = wids[woff[q]:woff[q + 1]]
        want = pay[hit].astype(np.int64).sum(0)
        assert cnt[q] == len(hit)
        assert np.array_equal(s[q], want.astype(np.float32))
        if len(hit):
            assert np.allclose(m[q], want / len(hit), rtol=1e-6, atol=0)
            assert np.allclose(dn[q] * np.pi * r2, want, rtol=1e-5, atol=1e-5)
        else:
            assert not m[q].any() and not dn[q].any()
    # kNN: over the k best, R^2 = the farthest found neighbour's d2
    k = 10
    ki, kd = oracle.knn_brute(pts, qs, k, 0.05)
    ks = oracle.knn_reduce(ki, kd, pay, oracle.REDUCE_SUM)
    kdn = oracle.knn_reduce(ki, kd, pay, oracle.REDUCE_DENSITY)
    for q in range(len(qs)):
        v = ki[q][ki[q] >= 0]
        want = pay[v].astype(np.int64).sum(0)
        assert np.array_equal(ks[q], want.astype(np.float32))
        if len(v):
            R2 = float(kd[q][len(v) - 1])
            assert R2 == float(kd[q][ki[q] >= 0].max())
            assert np.allclose(kdn[q] * np.pi * R2, want, rtol=1e-5, atol=1e-5)


def test_payload_reductions_of_empty_sets_are_zero():
    """A query with no hit reduces to 0 in every mode (no 0/0 for the mean, nor
    for the kNN density, whose disc has radius 0 when nothing was found)."""
    g = np.random.default_rng(19)
    N, C = 500, 3
    pts = g.random((N, 3)).astype(np.float32)
    pay = g.integers(1, 9, size=(N, C)).astype(np.float32)
    pid = oracle.build(pts)
    qs = np.array([[5.0, 5.0, 5.0], [-3.0, 0.5, 0.5], [0.5, 0.5, 9.0]], dtype=np.float32)
    for mode in (oracle.REDUCE_SUM, oracle.REDUCE_MEAN, oracle.REDUCE_DENSITY):
        out, cnt = oracle.range_reduce(pts, pid, qs, 0.25, pay, mode)
        assert cnt.tolist() == [0, 0, 0]
        assert np.array_equal(out, np.zeros((3, C), dtype=np.float32)), mode
        ki, kd = oracle.knn_brute(pts, qs, 4, 0.25)
        assert (ki == -1).all()
        assert np.array_equal(oracle.knn_reduce(ki, kd, pay, mode), np.zeros((3, C), dtype=np.float32)), mode


def test_payload_sum_float_within_rounding_bound():
    """Float payloads: the sequential FP32 sum is within n * eps * sum|x| of the FP64 sum."""
    g = np.random.default_rng(10)
    N, D, C = 2000, 2, 3
    pts = g.random((N, D)).astype(np.float32)
    pay = g.standard_normal((N, C)).astype(np.float32)
    pid = oracle.build(pts)
    qs = g.random((50, D)).astype(np.float32)
    s, cnt = oracle.range_reduce(pts, pid, qs, 0.1, pay, oracle.REDUCE_SUM)
    _, woff, wids, _ = oracle.radius_brute(pts, qs, 0.1)
    eps = np.finfo(np.float32).eps
    for q in range(len(qs)):
        x = pay[wids[woff[q]:woff[q + 1]]].astype(np.float64)
        bound = len(x) * eps * np.abs(x).sum(0) + 1e-30
        assert np.all(np.abs(s[q] - x.sum(0)) <= bound)


# ------------------------------------- swapped order (node after close subtree)

CLOSE_FIRST = 2


@pytest.mark.parametrize("seed", range(8))
def test_close_first_equals_brute_and_recursion(seed):
    """The footnote of Sec. 3.1 allows processing a node after its close
    subtree: the same exact results, and the stack-free machine walks the
    same steps as the recursion in that order."""
    g = np.random.default_rng(700 + seed)
    N, D = int(g.integers(1, 260)), int(g.integers(1, 5))
    pts = g.random((N, D)).astype(np.float32)
    if seed % 2:
        pts = g.integers(0, 4, size=(N, D)).astype(np.float32)
    pid = oracle.build(pts)
    qs = (g.random((12, D)) * 1.2 - 0.1).astype(np.float32)
    for k, r in ((1, math.inf), (4, math.inf), (8, 0.3), (N + 2, math.inf)):
        want_i, want_d = oracle.knn_brute(pts, qs, k, r)
        for i in range(len(qs)):
            a = oracle.knn_recursive(pts, pid, qs[i], k, r, ordered=CLOSE_FIRST)
            b = oracle.knn_stackfree(pts, pid, qs[i], k, r, ordered=CLOSE_FIRST)
            assert np.array_equal(a[0], want_i[i]) and np.array_equal(a[1].view(np.uint32), want_d[i].view(np.uint32))
            assert np.array_equal(b[0], a[0]) and np.array_equal(b[1], a[1])
            assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])
        got = oracle.knn_tree(pts, pid, qs, k, r, ordered=CLOSE_FIRST)
        assert np.array_equal(got[0], want_i) and np.array_equal(got[1], want_d)


def test_close_first_unbounded_is_inorder_by_close_side():
    """With k >= N and r = inf nothing is culled: every node is processed once,
    after all nodes of its close subtree and before all nodes of its far one."""
    g = np.random.default_rng(5)
    N, D = 200, 3
    pts = g.random((N, D)).astype(np.float32)
    pid = oracle.build(pts)
    q = g.random(D).astype(np.float32)

    def subtree(n):
        out, stack = [], [n]
        while stack:
            m = stack.pop()
            if m < N:
                out.append(m)
                stack += [2 * m + 1, 2 * m + 2]
        return out

    _, _, visits, _ = oracle.knn_stackfree(pts, pid, q, N, math.inf, ordered=CLOSE_FIRST)
    assert sorted(visits.tolist()) == list(range(N))
    pos = np.empty(N, dtype=np.int64)
    pos[visits] = np.arange(N)
    for n in range(N):
        d = int(np.floor(np.log2(n + 1))) % D
        sd = np.float32(q[d]) - pts[pid[n], d]
        close, far = (2 * n + 2, 2 * n + 1) if sd > 0 else (2 * n + 1, 2 * n + 2)
        assert all(pos[m] < pos[n] for m in subtree(close))
        assert all(pos[m] > pos[n] for m in subtree(far))


def test_close_first_six_point_trace():
    """Figure 1's points, query (8,1.5), k = 1: the root-first order processes
    (7,2) first; close-first descends to (8,1) before processing anything."""
    gd = json.load(open(GOLDEN))
    pts = np.array(gd["points"], dtype=np.float32)
    pid = oracle.build(pts)
    q = np.array([8.0, 1.5], dtype=np.float32)
    _, _, v_root, _ = oracle.knn_stackfree(pts, pid, q, 1)
    ids, _, v_close, _ = oracle.knn_stackfree(pts, pid, q, 1, ordered=CLOSE_FIRST)
    assert tuple(pts[pid[v_root[0]]].tolist()) == (7.0, 2.0)
    assert tuple(pts[pid[v_close[0]]].tolist()) == (8.0, 1.0)
    assert tuple(pts[ids[0]].tolist()) == (8.0, 1.0)


@pytest.mark.parametrize("seed", range(4))
def test_range_visits_equal_unordered_knn_with_unfillable_list(seed):
    """A ball query is the unordered kNN traversal whose list never fills
    (k > N): the cull radius stays r^2, so both process the same nodes."""
    g = np.random.default_rng(900 + seed)
    N, D = int(g.integers(1, 120)), int(g.integers(1, 4))
    pts = g.random((N, D)).astype(np.float32)
    if seed % 2:
        pts = g.integers(0, 4, size=(N, D)).astype(np.float32)
    pid = oracle.build(pts)
    qs = (g.random((30, D)) * 1.2 - 0.1).astype(np.float32)
    for r in (0.0, 0.15, 0.5, math.inf):
        v = oracle.range_visits(pts, pid, qs, radius=r)
        _, _, kv = oracle.knn_tree(pts, pid, qs, N + 1, r, ordered=False)
        assert np.array_equal(v, kv), r
    # r = inf processes every node once
    assert np.all(oracle.range_visits(pts, pid, qs, radius=math.inf) == N)


def test_radius_brute_against_fp64_up_to_boundary_ties():
    """The ball query's FP32 hit sets equal the FP64 definition except for points
    whose distance lies within a few float ulps of the radius."""
    g = np.random.default_rng(31)
    pts = g.random((4000, 3)).astype(np.float32)
    qs = g.random((50, 3)).astype(np.float32)
    r = 0.11
    counts, off, ids, d2 = oracle.radius_brute(pts, qs, r)
    r2_64 = float(np.float32(r) * np.float32(r))
    for q in range(len(qs)):
        d64 = ((pts.astype(np.float64) - qs[q].astype(np.float64)) ** 2).sum(1)
        want = set(np.nonzero(d64 <= r2_64)[0].tolist())
        got = set(ids[off[q]:off[q + 1]].tolist())
        for i in want ^ got:
            assert abs(d64[i] - r2_64) <= 8 * np.spacing(np.float32(r2_64)), (q, i)
