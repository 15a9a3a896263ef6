"""CPU oracle for the k-d tree queries of arXiv 2210.12859 (Wald).

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The CUDA library never imports, links
or loads anything from here.

The arithmetic lives in ``kdt_oracle.c`` (plain C, compiled with
``-O2 -ffp-contract=off``, no fast-math), this module only marshals numpy
arrays.  ``ensure_built()`` compiles the shared object when it is missing or
older than its source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# KDT_ORACLE_SRC points the module at another copy of the C source (the
# mutation tests compile deliberately broken copies and check that the pins
# reject each of them); the shared object is built next to that copy.
_SRC = os.path.abspath(os.environ.get("KDT_ORACLE_SRC") or os.path.join(_HERE, "kdt_oracle.c"))
_LIB = os.path.join(os.path.dirname(_SRC), "libkdt_oracle.so")
_lock = threading.Lock()
_lib = None

# gcc flags: every float operation evaluated as written (no contraction into
# fused multiply-add, which GCC does by default on aarch64), no fast-math.
CFLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread"]


def ensure_built(force: bool = False) -> str:
    """Compile ``libkdt_oracle.so`` next to its source if needed; return its path."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(ensure_built())
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        i32 = ctypes.c_int
        f32 = ctypes.c_float
        lib.orc_left_size.argtypes = [i64]
        lib.orc_left_size.restype = i64
        lib.orc_build.argtypes = [P, i64, i32, P]
        lib.orc_build.restype = i32
        lib.orc_radius_brute.argtypes = [P, i64, i32, P, i64, f32, P, P, P, P]
        lib.orc_radius_brute.restype = None
        lib.orc_box_brute.argtypes = [P, i64, i32, P, P, i64, P, P, P]
        lib.orc_box_brute.restype = None
        lib.orc_range_stackfree.argtypes = [P, P, P, i64, i32, i32, P, P, i64, f32, P, P, P, P]
        lib.orc_range_stackfree.restype = i32
        lib.orc_range_visits.argtypes = [P, P, P, i64, i32, i32, P, P, i64, f32, P]
        lib.orc_range_visits.restype = i32
        lib.orc_range_reduce.argtypes = [P, P, P, i64, i32, P, i64, f32, P, i32, i32, P, P]
        lib.orc_range_reduce.restype = i32
        lib.orc_knn_reduce.argtypes = [P, P, i64, i32, P, i32, i32, P]
        lib.orc_knn_reduce.restype = None
        lib.orc_build_widest.argtypes = [P, i64, i32, P, P]
        lib.orc_build_widest.restype = i32
        lib.orc_build_par.argtypes = [P, i64, i32, P, P, i32]
        lib.orc_build_par.restype = i32
        lib.orc_knn_stackfree_batch_dims.argtypes = [P, P, P, i64, i32, P, i64, i32, f32, i32, P, P, P]
        lib.orc_knn_stackfree_batch_dims.restype = i32
        lib.orc_knn_brute.argtypes = [P, i64, i32, P, i64, i32, f32, P, P]
        lib.orc_knn_brute.restype = None
        lib.orc_knn_brute_f64.argtypes = [P, i64, i32, P, i64, i32, P, P]
        lib.orc_knn_brute_f64.restype = None
        trav = [P, P, i64, i32, P, i32, f32, i32, P, P, P, i64, P, P, i64, P]
        lib.orc_knn_recursive.argtypes = trav
        lib.orc_knn_recursive.restype = i32
        lib.orc_knn_stackfree.argtypes = trav
        lib.orc_knn_stackfree.restype = i32
        lib.orc_knn_stackfree_batch.argtypes = [P, P, i64, i32, P, i64, i32, f32, i32, P, P, P]
        lib.orc_knn_stackfree_batch.restype = i32
        lib.orc_descent_leaf.argtypes = [P, P, P, i64, i32, P]
        lib.orc_descent_leaf.restype = f32
        lib.orc_round_bf16.argtypes = [f32]
        lib.orc_round_bf16.restype = f32
        lib.orc_mlp_forward.argtypes = [P, i32, P, i64, P]
        lib.orc_mlp_forward.restype = None
        lib.orc_mlp_forward_bound.argtypes = [P, i32, P, i64, P, P]
        lib.orc_mlp_forward_bound.restype = None
        lib.orc_mlp_loss_grad_bound.argtypes = [P, i32, P, P, i64, P, P]
        lib.orc_mlp_loss_grad_bound.restype = ctypes.c_double
        lib.orc_mlp_loss_grad.argtypes = [P, i32, P, P, i64, P]
        lib.orc_mlp_loss_grad.restype = ctypes.c_double
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def left_size(n: int) -> int:
    """Left-subtree size of the root of a complete tree with n nodes."""
    return int(_load().orc_left_size(int(n)))


def build(points, threads: int = 1) -> np.ndarray:
    """Level-order tree as node -> input index (int32[N]); threads > 1 builds
    the subtrees of the top levels in parallel (the same tree)."""
    pts = _f32(points)
    N, D = pts.shape
    out = np.empty(N, dtype=np.int32)
    lib = _load()
    rc = (lib.orc_build_par(_ptr(pts), N, D, _ptr(out), None, int(threads)) if threads > 1
          else lib.orc_build(_ptr(pts), N, D, _ptr(out)))
    if rc != 0:
        raise ValueError("oracle build failed (bad arguments or non-finite point)")
    return out


def build_widest(points, threads: int = 1):
    """Level-order tree with a stored split dimension per node (widest extent
    of the node's points): (node -> input index int32[N], dims uint8[N])."""
    pts = _f32(points)
    N, D = pts.shape
    out = np.empty(N, dtype=np.int32)
    dims = np.empty(N, dtype=np.uint8)
    lib = _load()
    rc = (lib.orc_build_par(_ptr(pts), N, D, _ptr(out), _ptr(dims), int(threads)) if threads > 1
          else lib.orc_build_widest(_ptr(pts), N, D, _ptr(out), _ptr(dims)))
    if rc != 0:
        raise ValueError("oracle build failed (bad arguments or non-finite point)")
    return out, dims


def knn_tree_dims(points, node_pid, node_dim, queries, k, max_radius=float("inf"), ordered=True):
    """Stack-free traversal of many queries over a tree with stored split
    dimensions: (ids, d2, first visits per query)."""
    pts, qs = _f32(points), _f32(queries)
    node_pid = np.ascontiguousarray(node_pid, dtype=np.int32)
    node_dim = np.ascontiguousarray(node_dim, dtype=np.uint8)
    N, D = pts.shape
    Q = qs.shape[0]
    ids = np.empty((Q, k), dtype=np.int32)
    d2 = np.empty((Q, k), dtype=np.float32)
    nv = np.empty(Q, dtype=np.int32)
    rc = _load().orc_knn_stackfree_batch_dims(_ptr(pts), _ptr(node_pid), _ptr(node_dim), N, D, _ptr(qs), Q, k,
                                              float(max_radius), int(ordered), _ptr(ids), _ptr(d2), _ptr(nv))
    if rc != 0:
        raise RuntimeError("oracle traversal exceeded its step cap")
    return ids, d2, nv


def knn_tree_threaded(points, node_pid, queries, k, max_radius=float("inf"), ordered=True, node_dim=None,
                      threads: int = 0):
    """The stack-free traversal of many queries (level mod D, or stored split
    dimensions with node_dim) split over host threads by query (each C call
    releases the GIL): (ids, d2, first visits per query)."""
    pts, qs = _f32(points), _f32(queries)
    node_pid = np.ascontiguousarray(node_pid, dtype=np.int32)
    dims = None if node_dim is None else np.ascontiguousarray(node_dim, dtype=np.uint8)
    N, D = pts.shape
    Q = qs.shape[0]
    threads = max(1, min(threads or (os.cpu_count() or 1), max(Q, 1)))
    ids = np.empty((Q, k), dtype=np.int32)
    d2 = np.empty((Q, k), dtype=np.float32)
    nv = np.empty(Q, dtype=np.int32)
    lib = _load()
    # interleaved chunks: expensive queries tend to sit together
    chunk = 64
    starts = list(range(0, Q, chunk))
    nxt = [0]
    lock = threading.Lock()
    failed = []

    def work():
        while True:
            with lock:
                if nxt[0] >= len(starts):
                    return
                a = starts[nxt[0]]
                nxt[0] += 1
            b = min(a + chunk, Q)
            sub = np.ascontiguousarray(qs[a:b])
            oi = np.empty((b - a, k), dtype=np.int32)
            od = np.empty((b - a, k), dtype=np.float32)
            ov = np.empty(b - a, dtype=np.int32)
            rc = lib.orc_knn_stackfree_batch_dims(_ptr(pts), _ptr(node_pid), None if dims is None else _ptr(dims), N,
                                                  D, _ptr(sub), b - a, k, float(max_radius), int(ordered), _ptr(oi),
                                                  _ptr(od), _ptr(ov))
            if rc != 0:
                failed.append(a)
            ids[a:b] = oi
            d2[a:b] = od
            nv[a:b] = ov

    ts = [threading.Thread(target=work) for _ in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if failed:
        raise RuntimeError("oracle traversal exceeded its step cap")
    return ids, d2, nv


def radius_brute(points, queries, radius: float):
    """Every point with d2 <= fl(r*r): (counts int32[Q], offsets int64[Q+1],
    ids int32[total], d2 float32[total]), ids of a query in index order."""
    pts, qs = _f32(points), _f32(queries)
    N, D = pts.shape
    Q = qs.shape[0]
    counts = np.empty(Q, dtype=np.int32)
    lib = _load()
    lib.orc_radius_brute(_ptr(pts), N, D, _ptr(qs), Q, float(radius), _ptr(counts), None, None, None)
    offsets = np.zeros(Q + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(counts)
    ids = np.empty(max(int(offsets[-1]), 1), dtype=np.int32)
    d2 = np.empty(max(int(offsets[-1]), 1), dtype=np.float32)
    lib.orc_radius_brute(_ptr(pts), N, D, _ptr(qs), Q, float(radius), _ptr(counts), _ptr(offsets), _ptr(ids),
                         _ptr(d2))
    return counts, offsets, ids[: offsets[-1]], d2[: offsets[-1]]


def box_brute(points, lo, hi):
    """Every point inside [lo, hi] (inclusive): (counts, offsets, ids)."""
    pts, lo, hi = _f32(points), _f32(lo), _f32(hi)
    N, D = pts.shape
    Q = lo.shape[0]
    counts = np.empty(Q, dtype=np.int32)
    lib = _load()
    lib.orc_box_brute(_ptr(pts), N, D, _ptr(lo), _ptr(hi), Q, _ptr(counts), None, None)
    offsets = np.zeros(Q + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(counts)
    ids = np.empty(max(int(offsets[-1]), 1), dtype=np.int32)
    lib.orc_box_brute(_ptr(pts), N, D, _ptr(lo), _ptr(hi), Q, _ptr(counts), _ptr(offsets), _ptr(ids))
    return counts, offsets, ids[: offsets[-1]]


def range_tree(points, node_pid, qa, qb=None, radius: float = 0.0, node_dim=None):
    """Ball (qb None, radius) or box ([qa, qb]) queries through the unordered
    stack-free machine: (counts, offsets, ids, d2 or None), hits in traversal order."""
    pts, qa = _f32(points), _f32(qa)
    N, D = pts.shape
    Q = qa.shape[0]
    kind = 0 if qb is None else 1
    qb = None if qb is None else _f32(qb)
    pid = np.ascontiguousarray(node_pid, dtype=np.int32)
    nd = None if node_dim is None else np.ascontiguousarray(node_dim, dtype=np.uint8)
    lib = _load()
    counts = np.empty(Q, dtype=np.int32)
    args = (_ptr(pts), _ptr(pid), None if nd is None else _ptr(nd), N, D, kind, _ptr(qa),
            None if qb is None else _ptr(qb), Q, float(radius))
    assert lib.orc_range_stackfree(*args, _ptr(counts), None, None, None) == 0
    offsets = np.zeros(Q + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(counts)
    ids = np.empty(max(int(offsets[-1]), 1), dtype=np.int32)
    d2 = np.empty(max(int(offsets[-1]), 1), dtype=np.float32) if kind == 0 else None
    assert lib.orc_range_stackfree(*args, _ptr(counts), _ptr(offsets), _ptr(ids),
                                   None if d2 is None else _ptr(d2)) == 0
    return counts, offsets, ids[: offsets[-1]], (None if d2 is None else d2[: offsets[-1]])


def range_visits(points, node_pid, qa, qb=None, radius: float = 0.0, node_dim=None):
    """Processed nodes of each ball (qb None) or box query's stack-free range traversal."""
    pts, qa = _f32(points), _f32(qa)
    N, D = pts.shape
    Q = qa.shape[0]
    qb = None if qb is None else _f32(qb)
    pid = np.ascontiguousarray(node_pid, dtype=np.int32)
    nd = None if node_dim is None else np.ascontiguousarray(node_dim, dtype=np.uint8)
    v = np.empty(Q, dtype=np.int32)
    assert _load().orc_range_visits(_ptr(pts), _ptr(pid), None if nd is None else _ptr(nd), N, D,
                                    0 if qb is None else 1, _ptr(qa), None if qb is None else _ptr(qb), Q,
                                    float(radius), _ptr(v)) == 0
    return v


REDUCE_SUM, REDUCE_MEAN, REDUCE_DENSITY = 0, 1, 2


def range_reduce(points, node_pid, queries, radius: float, payload, mode: int, node_dim=None):
    """Payload reductions over ball hits in traversal order: (out [Q][C], counts)."""
    pts, qs = _f32(points), _f32(queries)
    pl = _f32(payload)
    N, D = pts.shape
    Q, C = qs.shape[0], pl.shape[1]
    pid = np.ascontiguousarray(node_pid, dtype=np.int32)
    nd = None if node_dim is None else np.ascontiguousarray(node_dim, dtype=np.uint8)
    out = np.empty((Q, C), dtype=np.float32)
    counts = np.empty(Q, dtype=np.int32)
    assert _load().orc_range_reduce(_ptr(pts), _ptr(pid), None if nd is None else _ptr(nd), N, D, _ptr(qs), Q,
                                    float(radius), _ptr(pl), C, int(mode), _ptr(out), _ptr(counts)) == 0
    return out, counts


def knn_reduce(ids, d2, payload, mode: int):
    """Payload reductions over kNN lists (ascending, -1 empty), in list order: out [Q][C]."""
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    d2 = _f32(d2)
    pl = _f32(payload)
    Q, k = ids.shape
    C = pl.shape[1]
    out = np.empty((Q, C), dtype=np.float32)
    _load().orc_knn_reduce(_ptr(ids), _ptr(d2), Q, k, _ptr(pl), C, int(mode), _ptr(out))
    return out


def knn_brute(points, queries, k: int, max_radius: float = float("inf")):
    """Plain definition: k smallest (d2, id) with d2 <= r2, FP32 distances."""
    pts, qs = _f32(points), _f32(queries)
    N, D = pts.shape
    Q = qs.shape[0]
    ids = np.empty((Q, k), dtype=np.int32)
    d2 = np.empty((Q, k), dtype=np.float32)
    _load().orc_knn_brute(_ptr(pts), N, D, _ptr(qs), Q, k, float(max_radius), _ptr(ids), _ptr(d2))
    return ids, d2


def knn_brute_threaded(points, queries, k: int, max_radius: float = float("inf"), threads: int = 0):
    """``knn_brute`` split over host threads by query (the C call releases the GIL)."""
    pts, qs = _f32(points), _f32(queries)
    Q = qs.shape[0]
    threads = threads or (os.cpu_count() or 1)
    threads = max(1, min(threads, Q))
    ids = np.empty((Q, k), dtype=np.int32)
    d2 = np.empty((Q, k), dtype=np.float32)
    bounds = np.linspace(0, Q, threads + 1).astype(np.int64)
    lib = _load()
    N, D = pts.shape

    def work(a, b):
        if b > a:
            sub = np.ascontiguousarray(qs[a:b])
            oi = np.empty((b - a, k), dtype=np.int32)
            od = np.empty((b - a, k), dtype=np.float32)
            lib.orc_knn_brute(_ptr(pts), N, D, _ptr(sub), b - a, k, float(max_radius), _ptr(oi), _ptr(od))
            ids[a:b] = oi
            d2[a:b] = od

    ts = [threading.Thread(target=work, args=(int(bounds[i]), int(bounds[i + 1]))) for i in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return ids, d2


def knn_brute_f64(points, queries, k: int):
    """k smallest (d2, id) with distances of the FP32 inputs evaluated in FP64."""
    pts, qs = _f32(points), _f32(queries)
    N, D = pts.shape
    Q = qs.shape[0]
    ids = np.empty((Q, k), dtype=np.int32)
    d2 = np.empty((Q, k), dtype=np.float64)
    _load().orc_knn_brute_f64(_ptr(pts), N, D, _ptr(qs), Q, k, _ptr(ids), _ptr(d2))
    return ids, d2


def _traverse(fn, points, node_pid, q, k, max_radius, ordered, log_cap):
    pts = _f32(points)
    node_pid = np.ascontiguousarray(node_pid, dtype=np.int32)
    N, D = pts.shape
    qv = _f32(q).reshape(D)
    ids = np.empty(k, dtype=np.int32)
    d2 = np.empty(k, dtype=np.float32)
    visits = np.empty(log_cap, dtype=np.int32)
    steps = np.empty(4 * log_cap, dtype=np.int32)
    nv = ctypes.c_int64(0)
    ns = ctypes.c_int64(0)
    rc = fn(_ptr(pts), _ptr(node_pid), N, D, _ptr(qv), k, float(max_radius), int(ordered),
            _ptr(ids), _ptr(d2), _ptr(visits), log_cap, ctypes.byref(nv), _ptr(steps),
            4 * log_cap, ctypes.byref(ns))
    if rc != 0:
        raise RuntimeError("oracle traversal exceeded its step cap")
    if nv.value > log_cap or ns.value > 4 * log_cap:
        raise RuntimeError("visit log overflow; raise log_cap")
    return ids, d2, visits[: nv.value].copy(), steps[: ns.value].copy()


def knn_recursive(points, node_pid, q, k, max_radius=float("inf"), ordered=True, log_cap=None):
    """Recursive traversal of one query: (ids, d2, first-visit log, step log)."""
    cap = log_cap or (len(node_pid) + 8)
    return _traverse(_load().orc_knn_recursive, points, node_pid, q, k, max_radius, ordered, cap)


def knn_stackfree(points, node_pid, q, k, max_radius=float("inf"), ordered=True, log_cap=None):
    """Stack-free state machine for one query: (ids, d2, first-visit log, step log)."""
    cap = log_cap or (len(node_pid) + 8)
    return _traverse(_load().orc_knn_stackfree, points, node_pid, q, k, max_radius, ordered, cap)


def knn_tree(points, node_pid, queries, k, max_radius=float("inf"), ordered=True):
    """Stack-free traversal of many queries: (ids, d2, first visits per query)."""
    pts, qs = _f32(points), _f32(queries)
    node_pid = np.ascontiguousarray(node_pid, dtype=np.int32)
    N, D = pts.shape
    Q = qs.shape[0]
    ids = np.empty((Q, k), dtype=np.int32)
    d2 = np.empty((Q, k), dtype=np.float32)
    nv = np.empty(Q, dtype=np.int32)
    rc = _load().orc_knn_stackfree_batch(_ptr(pts), _ptr(node_pid), N, D, _ptr(qs), Q, k,
                                         float(max_radius), int(ordered), _ptr(ids), _ptr(d2), _ptr(nv))
    if rc != 0:
        raise RuntimeError("oracle traversal exceeded its step cap")
    return ids, d2, nv


def descent_leaf_d2(points, node_pid, queries, node_dim=None) -> np.ndarray:
    """FP32 squared distance to the point where the greedy close-child descent
    ends; node_dim: the split dimension stored per node (build_widest), else
    level mod D."""
    pts, qs = _f32(points), _f32(queries)
    node_pid = np.ascontiguousarray(node_pid, dtype=np.int32)
    N, D = pts.shape
    dims = None if node_dim is None else np.ascontiguousarray(node_dim, dtype=np.uint8)
    if dims is not None and dims.shape != (N,):
        raise ValueError("node_dim must hold one dimension per node")
    lib = _load()
    out = np.empty(qs.shape[0], dtype=np.float32)
    for i in range(qs.shape[0]):
        qi = np.ascontiguousarray(qs[i])
        out[i] = lib.orc_descent_leaf(_ptr(pts), _ptr(node_pid), None if dims is None else _ptr(dims), N, D,
                                      _ptr(qi))
    return out


def round_bf16(x: float) -> float:
    """Nearest bfloat16 value (ties to even) of a finite float, as float."""
    return float(_load().orc_round_bf16(float(x)))


def mlp_param_count(H: int) -> int:
    return H * 4 + H + H * H + H + H + 1


def mlp_forward(params, H: int, x) -> np.ndarray:
    """FP64 forward of the 4->H->H->1 ReLU MLP (params: W1,b1,W2,b2,w3,b3)."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    xs = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 4)
    y = np.empty(xs.shape[0], dtype=np.float64)
    _load().orc_mlp_forward(_ptr(p), H, _ptr(xs), xs.shape[0], _ptr(y))
    return y


def mlp_forward_bound(params, H: int, x):
    """FP64 forward of the model and, per sample, a bound on the error of an
    evaluation with BF16 hidden activations and FP32 arithmetic (any order,
    rounding or truncating): (y float64[n], bound float64[n])."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    xs = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(xs.shape[0], dtype=np.float64)
    bound = np.empty(xs.shape[0], dtype=np.float64)
    _load().orc_mlp_forward_bound(_ptr(p), H, _ptr(xs), xs.shape[0], _ptr(y), _ptr(bound))
    return y, bound


def mlp_loss_grad_bound(params, H: int, x, label):
    """FP64 loss and gradient of the model and, per parameter, a bound on the
    error of a BF16-in / FP32-accumulate evaluation: (loss, grad float64[P],
    bound float64[P], loss bound)."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    xs = np.ascontiguousarray(x, dtype=np.float64)
    lab = np.ascontiguousarray(label, dtype=np.float64)
    P = mlp_param_count(H)
    grad = np.empty(P, dtype=np.float64)
    bound = np.empty(P + 1, dtype=np.float64)
    loss = _load().orc_mlp_loss_grad_bound(_ptr(p), H, _ptr(xs), _ptr(lab), xs.shape[0], _ptr(grad), _ptr(bound))
    return loss, grad, bound[:P], bound[P]


def mlp_loss_grad(params, H: int, x, label):
    """FP64 mean-squared-error loss and its gradient w.r.t. all parameters."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    xs = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 4)
    lab = np.ascontiguousarray(label, dtype=np.float64).reshape(-1)
    g = np.empty_like(p)
    loss = _load().orc_mlp_loss_grad(_ptr(p), H, _ptr(xs), _ptr(lab), xs.shape[0], _ptr(g))
    return float(loss), g
