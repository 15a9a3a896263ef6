"""The size-independent tree checks that the GPU tests apply to large trees.

At sizes where the oracle's recursive builder is too slow, the GPU tests
check a built tree by its separation property instead (`kdt_checks`).  Here,
on the CPU, those checks must accept every tree the oracle builds (ties, -0,
duplicates, ragged last levels included) and reject trees with one planted
defect: two nodes exchanged, a repeated id, a wrong stored dimension.
"""
import numpy as np
import pytest

import oracle
from kdt_checks import check_tree, check_tree_widest, float_key


def _points(N, D, seed, kind):
    g = np.random.default_rng(seed)
    if kind == "ties":
        return g.integers(0, 3, size=(N, D)).astype(np.float32)
    if kind == "zeros":
        p = g.integers(-1, 2, size=(N, D)).astype(np.float32) * np.float32(0.0)  # +0 and -0
        p[:: 3] = g.random((len(p[:: 3]), D)).astype(np.float32)
        return p
    return g.random((N, D)).astype(np.float32)


CASES = [(N, D, s, kind) for s, (N, D) in enumerate([(1, 1), (2, 3), (7, 2), (64, 3), (100, 4), (257, 8), (1000, 3)])
         for kind in ("random", "ties", "zeros")]


@pytest.mark.parametrize("N,D,seed,kind", CASES)
def test_check_tree_accepts_oracle_trees(N, D, seed, kind):
    pts = _points(N, D, seed, kind)
    pid = oracle.build(pts)
    check_tree(pts, pid, pts[pid])


@pytest.mark.parametrize("N,D,seed,kind", [c for c in CASES if c[0] >= 7])
def test_check_tree_rejects_planted_defects(N, D, seed, kind):
    pts = _points(N, D, seed, kind)
    pid = oracle.build(pts)
    g = np.random.default_rng(seed + 50)
    # the separation property determines the tree, so exchanging any two
    # nodes must be rejected, even two points with equal coordinates (their
    # indices still order them)
    for _ in range(20):
        a, b = (int(x) for x in g.choice(N, size=2, replace=False))
        bad = pid.copy()
        bad[a], bad[b] = bad[b], bad[a]
        with pytest.raises(AssertionError):
            check_tree(pts, bad)
    dup = pid.copy()
    dup[-1] = dup[0]
    with pytest.raises(AssertionError):
        check_tree(pts, dup)
    with pytest.raises(AssertionError):
        check_tree(pts, pid, pts[pid][::-1].copy())


@pytest.mark.parametrize("N,D,seed,kind", [c for c in CASES if c[1] <= 3])
def test_check_tree_widest_accepts_oracle_trees_and_rejects_defects(N, D, seed, kind):
    pts = _points(N, D, seed, kind)
    pid, dims = oracle.build_widest(pts)
    check_tree_widest(pts, pid, dims)
    if N < 7:
        return
    g = np.random.default_rng(seed + 60)
    a, b = (int(x) for x in g.choice(N, size=2, replace=False))
    bad = pid.copy()
    bad[a], bad[b] = bad[b], bad[a]
    with pytest.raises(AssertionError):
        check_tree_widest(pts, bad, dims)
    if D > 1:
        wrong = dims.copy()
        wrong[0] = (wrong[0] + 1) % D
        with pytest.raises(AssertionError):
            check_tree_widest(pts, pid, wrong)


def test_float_key_orders_like_floats():
    g = np.random.default_rng(7)
    x = np.concatenate([np.array([0.0, -0.0, 1e-45, -1e-45, 3.4e38, -3.4e38], dtype=np.float32),
                        (g.standard_normal(500) * 10.0 ** g.integers(-20, 20, 500)).astype(np.float32)])
    k = float_key(x)
    o = np.argsort(x, kind="stable")
    assert np.all((x[o][1:] > x[o][:-1]) == (k[o][1:] > k[o][:-1]))
    assert np.all((x[o][1:] == x[o][:-1]) == (k[o][1:] == k[o][:-1]))
