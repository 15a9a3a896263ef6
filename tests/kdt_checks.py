"""Test-side checks that hold at any size (no oracle arithmetic)."""
import numpy as np


def float_key(x: np.ndarray) -> np.ndarray:
    """Order-preserving uint64 key of float32 values (-0 sorts as +0)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = np.where(u == 0x80000000, 0, u)
    neg = (u & 0x80000000) != 0
    return np.where(neg, (~u) & 0xFFFFFFFF, u | 0x80000000)


def check_tree(points: np.ndarray, node_ids: np.ndarray, node_coords: np.ndarray | None = None) -> None:
    """Assert that node_ids is the level-order left-balanced k-d tree of the
    points with split dimension (level mod D) and (coordinate, index) order:
    the ids form a permutation, and every node's key in its split dimension is
    above every key of its left subtree and below every key of its right
    subtree.  Those conditions determine the tree uniquely."""
    N, D = points.shape
    ids = np.asarray(node_ids, dtype=np.int64)
    assert ids.shape == (N,)
    assert np.array_equal(np.sort(ids), np.arange(N)), "ids are not a permutation"
    if node_coords is not None:
        assert np.array_equal(np.asarray(node_coords).view(np.uint32), points[ids].view(np.uint32))
    H = int(np.floor(np.log2(N)))
    lvl_start = [(1 << l) - 1 for l in range(H + 2)]
    for d in range(D):
        key = (float_key(points[ids, d]) << np.uint64(32)) | ids.astype(np.uint64)
        mn = key.copy()
        mx = key.copy()
        for l in range(H - 1, -1, -1):
            t = np.arange(lvl_start[l], min(lvl_start[l + 1], N))
            for c in (2 * t + 1, 2 * t + 2):
                ok = c < N
                tt, cc = t[ok], c[ok]
                mn[tt] = np.minimum(mn[tt], mn[cc])
                mx[tt] = np.maximum(mx[tt], mx[cc])
        for l in range(0, H + 1):
            if l % D != d:
                continue
            t = np.arange(lvl_start[l], min(lvl_start[l + 1], N))
            lc, rc = 2 * t + 1, 2 * t + 2
            okl, okr = lc < N, rc < N
            assert (mx[lc[okl]] < key[t[okl]]).all(), f"left subtree not below its node (level {l})"
            assert (key[t[okr]] < mn[rc[okr]]).all(), f"right subtree not above its node (level {l})"


def check_tree_widest(points: np.ndarray, node_ids: np.ndarray, node_dims: np.ndarray) -> None:
    """As check_tree, for trees whose split dimension is stored per node: each
    stored dimension is the widest extent (max - min in float32, ties to the
    lowest index) of the node's subtree points, and the node separates its
    subtrees in that dimension under the (coordinate, index) order."""
    N, D = points.shape
    ids = np.asarray(node_ids, dtype=np.int64)
    dims = np.asarray(node_dims, dtype=np.int64)
    assert np.array_equal(np.sort(ids), np.arange(N)), "ids are not a permutation"
    H = int(np.floor(np.log2(N)))
    lvl_start = [(1 << l) - 1 for l in range(H + 2)]
    c = points[ids]
    lo, hi = c.copy(), c.copy()
    keys = [(float_key(c[:, d]) << np.uint64(32)) | ids.astype(np.uint64) for d in range(D)]
    mn = [k.copy() for k in keys]
    mx = [k.copy() for k in keys]
    for l in range(H - 1, -1, -1):
        t = np.arange(lvl_start[l], min(lvl_start[l + 1], N))
        for ch in (2 * t + 1, 2 * t + 2):
            ok = ch < N
            tt, cc = t[ok], ch[ok]
            lo[tt] = np.minimum(lo[tt], lo[cc])
            hi[tt] = np.maximum(hi[tt], hi[cc])
            for d in range(D):
                mn[d][tt] = np.minimum(mn[d][tt], mn[d][cc])
                mx[d][tt] = np.maximum(mx[d][tt], mx[d][cc])
    ext = (hi - lo).astype(np.float32)
    assert np.array_equal(dims, np.argmax(ext, axis=1)), "stored dimension is not the widest extent"
    t = np.arange(N)
    lc, rc = 2 * t + 1, 2 * t + 2
    for d in range(D):
        sel = dims == d
        okl = sel & (lc < N)
        okr = sel & (rc < N)
        assert (mx[d][lc[okl]] < keys[d][t[okl]]).all(), "left subtree not below its node"
        assert (keys[d][t[okr]] < mn[d][rc[okr]]).all(), "right subtree not above its node"
