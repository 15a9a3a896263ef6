"""Index identities the traversal kernels rely on, checked by enumeration.

In the level-order tree of Sec. 3 (children 2i+1 and 2i+2) the leftmost
descendant of node i that lies m levels below it is 2^m (i + 1) - 1.  The
kNN and range kernels decide whether a node's whole subtree fits in one step
by comparing i with floor(N / 2^m) instead of forming that index (which can
overflow 32 bits near N = 2^30): the descendant exists, i.e. 2^m (i + 1) - 1
< N, exactly when i < floor(N / 2^m).  Checked here for every i of every N up
to 3000 and on random indices up to the library's size limit 2^30 - 1.
"""
import numpy as np


def leftmost_descendant(i: int, m: int) -> int:
    node = i
    for _ in range(m):
        node = 2 * node + 1  # walk down the left children one level at a time
    return node


def test_threshold_equals_descendant_existence_small():
    for N in range(1, 3001):
        for m in range(1, 6):
            thr = N >> m
            for i in range(N):
                assert (leftmost_descendant(i, m) < N) == (i < thr), (N, m, i)


def test_threshold_equals_descendant_existence_large():
    g = np.random.default_rng(7)
    for N in list(g.integers(1 << 20, 1 << 30, 64)) + [(1 << 30) - 1, 1 << 29, (1 << 29) + 1]:
        N = int(N)
        for m in range(1, 6):
            thr = N >> m
            cand = [0, thr - 1, thr, thr + 1, N - 1] + [int(x) for x in g.integers(0, N, 32)]
            for i in cand:
                if 0 <= i < N:
                    assert (leftmost_descendant(i, m) < N) == (i < thr), (N, m, i)


def test_children_of_a_node_share_a_sector_with_the_one_slot_offset():
    """Nodes are stored one 16-byte slot in, so node j sits in slot j + 1 and
    the siblings 2i+1, 2i+2 (slots 2i+2, 2i+3) share one 32-byte sector, as do
    four consecutive grandchildren of one node in two sectors."""
    for i in range(0, 5000):
        l, r = 2 * i + 1, 2 * i + 2
        assert (l + 1) // 2 == (r + 1) // 2
        g = [2 * l + 1, 2 * l + 2, 2 * r + 1, 2 * r + 2]
        assert len({(x + 1) // 2 for x in g}) == 2
