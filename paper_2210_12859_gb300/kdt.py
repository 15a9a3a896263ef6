"""Python binding of the C ABI in include/kdt.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  Device
arrays are torch CUDA tensors (torch supplies device memory and streams, no
compute); host arrays are numpy arrays or CPU tensors.  The library is
``libkdt.so`` built in-tree by ``build.py``; importing this module without it
raises, there is no fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkdt.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")

_lib = ctypes.CDLL(LIB_PATH)

KDT_OK = 0
KDT_EINVAL = -1
KDT_ENONFINITE = -2
KDT_ENOMEM = -3
KDT_ECUDA = -4
KDT_ETRAVERSAL = -5
KDT_ENOMODEL = -6
KDT_EIO = -7

KDT_ORDERED = 0x0
KDT_UNORDERED = 0x1
KDT_MORTON = 0x2
KDT_LEARNED = 0x4
KDT_NO_STAGE = 0x8
KDT_PER_TREE = 0x10
KDT_COST_ORDER = 0x20
KDT_PLAIN_STEP = 0x40
KDT_CLOSE_FIRST = 0x80
KDT_STACK = 0x100
KDT_RANGE_VISITS = 0x200
KDT_BUILD_ASYNC = 0x1
KDT_REDUCE_SUM, KDT_REDUCE_MEAN, KDT_REDUCE_DENSITY = 0, 1, 2
KDT_PAYLOAD_MAX_C = 8
KDT_BUILD_WIDEST = 0x2
KDT_GATE_AUTO, KDT_GATE_ALL, KDT_GATE_FAR, KDT_GATE_NONE = 0, 1, 2, 3

MLP_HIDDEN = 64
MLP_PARAMS = 64 * 4 + 64 + 64 * 64 + 64 + 64 + 1


class KdtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_F = ctypes.c_float
_D = ctypes.c_double


class TrainOpts(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("margin", ctypes.c_float), ("fallback_target", ctypes.c_float),
                ("uniform_weights", ctypes.c_int), ("gate", ctypes.c_int), ("query_flags", ctypes.c_int)]


def _sig(name, args, res=_I):
    fn = getattr(_lib, name)
    fn.argtypes = args
    fn.restype = res
    return fn


_lib.kdt_last_error.restype = ctypes.c_char_p
_sig("kdt_launch_count", [], _I64)
_sig("kdt_build", [_P, _I64, _I, _P, ctypes.POINTER(_P)])
_sig("kdt_build_ex", [_P, _I64, _I, _I, _P, ctypes.POINTER(_P)])
_sig("kdt_rebuild", [_P, _P, _I, _P])
_sig("kdt_tree_info", [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I)])
_sig("kdt_tree_export", [_P, _P, _P, _P])
_sig("kdt_tree_save", [_P, ctypes.c_char_p])
_sig("kdt_tree_split_dims", [_P, _P, _P])
_sig("kdt_tree_load", [ctypes.c_char_p, _P, ctypes.POINTER(_P)])
_sig("kdt_fcp", [_P, _P, _I64, _F, _I, _P, _P, _P])
_sig("kdt_knn", [_P, _P, _I64, _I, _F, _I, _P, _P, _P])
_sig("kdt_knn_visits", [_P, _P, _I64, _I, _F, _I, _P, _P])
_sig("kdt_knn_static", [_P, _P, _I64, _I, _F, _I, _P, _P, _P])
_sig("kdt_radius_count", [_P, _P, _I64, _F, _I, _P, _P])
_sig("kdt_radius_fill", [_P, _P, _I64, _F, _I, _P, _P, _P, _P])
_sig("kdt_box_count", [_P, _P, _P, _I64, _I, _P, _P])
_sig("kdt_box_fill", [_P, _P, _P, _I64, _I, _P, _P, _P])
_sig("kdt_offsets", [_P, _I64, _P, ctypes.POINTER(_I64), _P])
_sig("kdt_tree_set_payload", [_P, _P, _I, _P])
_sig("kdt_radius_reduce", [_P, _P, _I64, _F, _I, _I, _P, _P, _P])
_sig("kdt_knn_reduce", [_P, _P, _I64, _I, _F, _I, _I, _P, _P])
_sig("kdt_status", [_P, _P])
_sig("kdt_free", [_P], None)
_sig("kdt_knn_host", [_P, _I64, _I, _P, _I64, _I, _F, _I, _P, _P])
_sig("kdt_build_batched", [_P, _P, _I, _I, _P, ctypes.POINTER(_P)])
_sig("kdt_knn_batched", [_P, _P, _P, _I, _F, _I, _P, _P, _P])
_sig("kdt_forest_export", [_P, _P, _P, _P])
_sig("kdt_forest_free", [_P], None)
_sig("kdt_forest_set_launch", [_P, _I, _I, _I, _I])
_sig("kdt_knn_batched_visits", [_P, _P, _P, _I, _F, _I, _P, _P])
_sig("kdt_forest_autotune", [_P, _P, _P, _I, _F, _I, _P, _P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                              ctypes.POINTER(_I), ctypes.POINTER(_F), _P])
_sig("kdt_profile_enable", [_P, _I])
_sig("kdt_debug_fail_allocs", [_I])
_sig("kdt_debug_set_step_cap", [_P, ctypes.c_uint32])
_sig("kdt_set_stage_levels", [_P, _I])
_sig("kdt_set_claim_steps", [_P, _I])
_sig("kdt_set_inline_depth", [_P, _I])
_sig("kdt_set_light_run", [_P, _I])
_sig("kdt_set_large_k_list", [_P, _I])
_sig("kdt_large_k_list", [_P, _I, _P])
_sig("kdt_tuned_params", [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)])
_sig("kdt_autotune", [_P, _P, _I64, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_F), _P])
_sig("kdt_tuning_save", [ctypes.c_char_p])
_sig("kdt_tuning_load", [ctypes.c_char_p])
_sig("kdt_profile_read", [_P, ctypes.POINTER(_D), ctypes.POINTER(_I64)])
_sig("kdt_l2_read_bandwidth", [_I64, _I, ctypes.POINTER(_D), _P])

_OPTIONAL = {}


def _optional(name, args, res=_I):
    try:
        _OPTIONAL[name] = _sig(name, args, res)
    except AttributeError:
        _OPTIONAL[name] = None


_optional("kdt_radius_model_train", [_P, _P, _I64, _I, ctypes.POINTER(TrainOpts), ctypes.POINTER(_F), _P])
_optional("kdt_radius_model_get", [_P, _P, _P, ctypes.POINTER(_F)])
_optional("kdt_radius_model_set", [_P, _P, _P, _F])
_optional("kdt_radius_model_save", [_P, ctypes.c_char_p])
_optional("kdt_radius_model_load", [_P, ctypes.c_char_p])
_optional("kdt_descent_features", [_P, _P, _I64, _P, _P])
_optional("kdt_mlp_forward", [_P, _P, _I64, _P, _P])
_optional("kdt_mlp_loss_grad", [_P, _P, _P, _I64, ctypes.POINTER(_F), _P, _P])
_optional("kdt_learned_stats", [_P, ctypes.POINTER(_I64), ctypes.POINTER(_D), _P])
_optional("kdt_learned_gated", [_P, ctypes.POINTER(_I64), _P])
_optional("kdt_radius_model_gate", [_P, ctypes.POINTER(_I)])
_optional("kdt_radius_model_set_gate", [_P, _I])


def _check(rc: int):
    if rc != KDT_OK:
        raise KdtError(rc, _lib.kdt_last_error().decode(errors="replace"))


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor, dtype, name: str, shape=None) -> ctypes.c_void_p:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _host(a, dtype, name: str) -> tuple:
    if isinstance(a, torch.Tensor):
        if a.is_cuda:
            raise TypeError(f"{name} must be a host array")
        if a.dtype != {np.float32: torch.float32, np.int32: torch.int32}[dtype]:
            raise TypeError(f"{name} must be {np.dtype(dtype).name}, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return ctypes.c_void_p(arr.ctypes.data), arr


def _host_out(a, dtype, name: str, shape) -> ctypes.c_void_p:
    """An output host array is written in place: it must already have the
    dtype, shape and contiguous layout (no converted copy to lose results in)."""
    if isinstance(a, torch.Tensor):
        p, t = _host(a, dtype, name)
    else:
        if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"{name} must be a C-contiguous {np.dtype(dtype).name} array")
        p, t = ctypes.c_void_p(a.ctypes.data), a
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return p


class Tree:
    """A library-owned tree (``kdt_tree*``); freed with ``kdt_free``."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle
        n = _I64()
        d = _I()
        _check(_lib.kdt_tree_info(handle, ctypes.byref(n), ctypes.byref(d)))
        self.N, self.D = n.value, d.value

    @property
    def handle(self):
        if not self._h:
            raise ValueError("tree was freed")
        return self._h

    def free(self):
        if self._h:
            _lib.kdt_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Forest:
    def __init__(self, handle, offsets: np.ndarray, D: int):
        self._h = handle
        self.offsets = offsets
        self.T = len(offsets) - 1
        self.D = D

    @property
    def handle(self):
        if not self._h:
            raise ValueError("forest was freed")
        return self._h

    def free(self):
        if self._h:
            _lib.kdt_forest_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ---------------------------------------------------------------- single tree

def kdt_build(points: torch.Tensor, opts: int = 0, stream=None) -> Tree:
    if points.dim() != 2:
        raise ValueError("points must be [N, D]")
    N, D = points.shape
    h = _P()
    _check(_lib.kdt_build_ex(_dev(points, torch.float32, "points"), N, D, opts, _stream(stream), ctypes.byref(h)))
    return Tree(h)


def kdt_build_ex(points: torch.Tensor, opts: int = 0, stream=None) -> Tree:
    return kdt_build(points, opts, stream)


def kdt_tree_info(tree: Tree):
    return tree.N, tree.D


def kdt_last_error() -> str:
    return _lib.kdt_last_error().decode(errors="replace")


def kdt_launch_count() -> int:
    return int(_lib.kdt_launch_count())


def kdt_rebuild(tree: Tree, points: torch.Tensor, opts: int = 0, stream=None) -> None:
    _dev(points, torch.float32, "points", (tree.N, tree.D))
    _check(_lib.kdt_rebuild(tree.handle, ctypes.c_void_p(points.data_ptr()), opts, _stream(stream)))
    tree.payload_c = 0  # the library drops a payload on rebuild


def kdt_tree_export(tree: Tree, stream=None):
    coords = torch.empty((tree.N, tree.D), dtype=torch.float32, device="cuda")
    ids = torch.empty(tree.N, dtype=torch.int32, device="cuda")
    _check(_lib.kdt_tree_export(tree.handle, ctypes.c_void_p(coords.data_ptr()), ctypes.c_void_p(ids.data_ptr()),
                                _stream(stream)))
    return coords, ids


def kdt_tree_split_dims(tree: Tree, stream=None) -> torch.Tensor:
    dims = torch.empty(tree.N, dtype=torch.uint8, device="cuda")
    _check(_lib.kdt_tree_split_dims(tree.handle, ctypes.c_void_p(dims.data_ptr()), _stream(stream)))
    return dims


def kdt_tree_save(tree: Tree, path: str) -> None:
    _check(_lib.kdt_tree_save(tree.handle, os.fsencode(path)))


def kdt_tree_load(path: str, stream=None) -> Tree:
    h = _P()
    _check(_lib.kdt_tree_load(os.fsencode(path), _stream(stream), ctypes.byref(h)))
    return Tree(h)


def _outputs(Q, k, out_ids, out_d2, dev):
    if out_ids is None:
        out_ids = torch.empty((Q, k), dtype=torch.int32, device=dev)
    if out_d2 is None:
        out_d2 = torch.empty((Q, k), dtype=torch.float32, device=dev)
    return out_ids, out_d2


def kdt_knn(tree: Tree, queries: torch.Tensor, k: int, max_radius: float = math.inf, flags: int = 0,
            out_ids=None, out_d2=None, stream=None):
    Q = queries.shape[0]
    out_ids, out_d2 = _outputs(Q, k, out_ids, out_d2, queries.device)
    _check(_lib.kdt_knn(tree.handle, _dev(queries, torch.float32, "queries", (Q, tree.D)), Q, k, float(max_radius),
                        flags, _dev(out_ids, torch.int32, "out_ids", (Q, k)),
                        _dev(out_d2, torch.float32, "out_d2", (Q, k)), _stream(stream)))
    return out_ids, out_d2


KDT_STATIC_MAX_Q = 1 << 18


def kdt_knn_static(tree: Tree, queries: torch.Tensor, k: int, max_radius: float = math.inf, flags: int = 0,
                   out_ids=None, out_d2=None, stream=None):
    """kdt_knn with its scratch in the library's fixed device array (no
    device allocation inside the call; Q <= KDT_STATIC_MAX_Q)."""
    Q = queries.shape[0]
    out_ids, out_d2 = _outputs(Q, k, out_ids, out_d2, queries.device)
    _check(_lib.kdt_knn_static(tree.handle, _dev(queries, torch.float32, "queries", (Q, tree.D)), Q, k,
                               float(max_radius), flags, _dev(out_ids, torch.int32, "out_ids", (Q, k)),
                               _dev(out_d2, torch.float32, "out_d2", (Q, k)), _stream(stream)))
    return out_ids, out_d2


def kdt_fcp(tree: Tree, queries: torch.Tensor, max_radius: float = math.inf, flags: int = 0,
            out_ids=None, out_d2=None, stream=None):
    Q = queries.shape[0]
    if out_ids is None:
        out_ids = torch.empty(Q, dtype=torch.int32, device=queries.device)
    if out_d2 is None:
        out_d2 = torch.empty(Q, dtype=torch.float32, device=queries.device)
    _check(_lib.kdt_fcp(tree.handle, _dev(queries, torch.float32, "queries", (Q, tree.D)), Q, float(max_radius),
                        flags, _dev(out_ids, torch.int32, "out_ids"), _dev(out_d2, torch.float32, "out_d2"),
                        _stream(stream)))
    return out_ids, out_d2


def kdt_knn_visits(tree: Tree, queries: torch.Tensor, k: int, max_radius: float = math.inf, flags: int = 0,
                   stream=None) -> torch.Tensor:
    Q = queries.shape[0]
    v = torch.empty(Q, dtype=torch.int32, device=queries.device)
    _check(_lib.kdt_knn_visits(tree.handle, _dev(queries, torch.float32, "queries", (Q, tree.D)), Q, k,
                               float(max_radius), flags, ctypes.c_void_p(v.data_ptr()), _stream(stream)))
    return v


def kdt_radius_count(tree: Tree, queries: torch.Tensor, radius: float, flags: int = 0,
                     stream=None) -> torch.Tensor:
    Q = queries.shape[0]
    counts = torch.empty(Q, dtype=torch.int32, device=queries.device)
    _check(_lib.kdt_radius_count(tree.handle, _dev(queries, torch.float32, "queries", (Q, tree.D)), Q, float(radius),
                                 flags, ctypes.c_void_p(counts.data_ptr()), _stream(stream)))
    return counts


def kdt_offsets(counts: torch.Tensor, stream=None):
    """Exclusive prefix offsets [Q+1] (int64) of the counts and their total."""
    Q = counts.shape[0]
    off = torch.empty(Q + 1, dtype=torch.int64, device=counts.device)
    total = _I64()
    _check(_lib.kdt_offsets(_dev(counts, torch.int32, "counts"), Q, ctypes.c_void_p(off.data_ptr()),
                            ctypes.byref(total), _stream(stream)))
    return off, total.value


def kdt_radius_fill(tree: Tree, queries: torch.Tensor, radius: float, offsets: torch.Tensor, total: int,
                    with_d2: bool = True, flags: int = 0, stream=None):
    Q = queries.shape[0]
    ids = torch.empty(max(total, 1), dtype=torch.int32, device=queries.device)
    d2 = torch.empty(max(total, 1), dtype=torch.float32, device=queries.device) if with_d2 else None
    _check(_lib.kdt_radius_fill(tree.handle, _dev(queries, torch.float32, "queries", (Q, tree.D)), Q, float(radius),
                                flags, _dev(offsets, torch.int64, "offsets", (Q + 1,)),
                                ctypes.c_void_p(ids.data_ptr()),
                                ctypes.c_void_p(d2.data_ptr()) if with_d2 else None, _stream(stream)))
    return ids[:total], (d2[:total] if with_d2 else None)


def kdt_radius_search(tree: Tree, queries: torch.Tensor, radius: float, flags: int = 0, stream=None):
    """All points within `radius` of each query: (offsets [Q+1], ids, d2)."""
    counts = kdt_radius_count(tree, queries, radius, flags, stream)
    off, total = kdt_offsets(counts, stream)
    ids, d2 = kdt_radius_fill(tree, queries, radius, off, total, True, flags, stream)
    return off, ids, d2


def kdt_box_count(tree: Tree, lo: torch.Tensor, hi: torch.Tensor, flags: int = 0, stream=None) -> torch.Tensor:
    Q = lo.shape[0]
    counts = torch.empty(Q, dtype=torch.int32, device=lo.device)
    _check(_lib.kdt_box_count(tree.handle, _dev(lo, torch.float32, "lo", (Q, tree.D)),
                              _dev(hi, torch.float32, "hi", (Q, tree.D)), Q, flags,
                              ctypes.c_void_p(counts.data_ptr()), _stream(stream)))
    return counts


def kdt_box_fill(tree: Tree, lo: torch.Tensor, hi: torch.Tensor, offsets: torch.Tensor, total: int, flags: int = 0,
                 stream=None):
    Q = lo.shape[0]
    ids = torch.empty(max(total, 1), dtype=torch.int32, device=lo.device)
    _check(_lib.kdt_box_fill(tree.handle, _dev(lo, torch.float32, "lo", (Q, tree.D)),
                             _dev(hi, torch.float32, "hi", (Q, tree.D)), Q, flags,
                             _dev(offsets, torch.int64, "offsets", (Q + 1,)), ctypes.c_void_p(ids.data_ptr()),
                             _stream(stream)))
    return ids[:total]


def kdt_box_search(tree: Tree, lo: torch.Tensor, hi: torch.Tensor, flags: int = 0, stream=None):
    """All points inside each box [lo, hi]: (offsets [Q+1], ids)."""
    counts = kdt_box_count(tree, lo, hi, flags, stream)
    off, total = kdt_offsets(counts, stream)
    return off, kdt_box_fill(tree, lo, hi, off, total, flags, stream)


def kdt_tree_set_payload(tree: Tree, payload: torch.Tensor, stream=None) -> None:
    """Attach a per-point payload float32 [N, C] (input order, 1 <= C <= 8)."""
    if payload.dim() != 2:
        raise ValueError("payload must be [N, C]")
    C = payload.shape[1]
    _check(_lib.kdt_tree_set_payload(tree.handle, _dev(payload, torch.float32, "payload", (tree.N, C)), C,
                                     _stream(stream)))
    tree.payload_c = C


def kdt_radius_reduce(tree: Tree, queries: torch.Tensor, radius: float, mode: int = 0, flags: int = 0,
                      with_counts: bool = False, stream=None):
    """Payload reduction over each ball's hits: out [Q, C] (and counts [Q])."""
    Q = queries.shape[0]
    C = getattr(tree, "payload_c", 0) or 1
    out = torch.empty((Q, C), dtype=torch.float32, device=queries.device)
    counts = torch.empty(Q, dtype=torch.int32, device=queries.device) if with_counts else None
    _check(_lib.kdt_radius_reduce(tree.handle, _dev(queries, torch.float32, "queries", (Q, tree.D)), Q,
                                  float(radius), flags, mode, ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(counts.data_ptr()) if with_counts else None, _stream(stream)))
    return (out, counts) if with_counts else out


def kdt_knn_reduce(tree: Tree, queries: torch.Tensor, k: int, max_radius: float = math.inf, mode: int = 0,
                   flags: int = 0, stream=None) -> torch.Tensor:
    """Payload reduction over each query's k nearest neighbours: out [Q, C]."""
    Q = queries.shape[0]
    C = getattr(tree, "payload_c", 0) or 1
    out = torch.empty((Q, C), dtype=torch.float32, device=queries.device)
    _check(_lib.kdt_knn_reduce(tree.handle, _dev(queries, torch.float32, "queries", (Q, tree.D)), Q, k,
                               float(max_radius), flags, mode, ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def kdt_status(tree: Tree, stream=None) -> None:
    _check(_lib.kdt_status(tree.handle, _stream(stream)))


def kdt_free(tree: Tree) -> None:
    tree.free()


def kdt_knn_host(points, queries, k: int, max_radius: float = math.inf, flags: int = 0, out_ids=None, out_d2=None):
    """Host-to-host kNN: host inputs in, host results out (one synchronous call)."""
    pp, pk = _host(points, np.float32, "points")
    qp, qk = _host(queries, np.float32, "queries")
    N, D = pk.shape
    Q = qk.shape[0]
    if out_ids is None:
        out_ids = np.empty((Q, k), dtype=np.int32)
    if out_d2 is None:
        out_d2 = np.empty((Q, k), dtype=np.float32)
    if Q > 0 and (qk.ndim != 2 or qk.shape[1] != D):
        raise ValueError(f"queries must be [Q, {D}]")
    ip = _host_out(out_ids, np.int32, "out_ids", (Q, k))
    dp = _host_out(out_d2, np.float32, "out_d2", (Q, k))
    _check(_lib.kdt_knn_host(pp, N, D, qp, Q, k, float(max_radius), flags, ip, dp))
    return out_ids, out_d2


def kdt_set_claim_steps(tree: Tree, steps: int) -> None:
    _check(_lib.kdt_set_claim_steps(tree.handle, steps))


def kdt_set_inline_depth(tree: Tree, depth: int) -> None:
    _check(_lib.kdt_set_inline_depth(tree.handle, depth))


def kdt_set_light_run(tree: Tree, steps: int) -> None:
    _check(_lib.kdt_set_light_run(tree.handle, steps))


KDT_LIST_SHARED, KDT_LIST_GLOBAL, KDT_LIST_GROUP4, KDT_LIST_GROUP8 = 0, 1, 2, 3


def kdt_set_large_k_list(tree: Tree, placement: int) -> None:
    """Where the k-best lists of k > 16 live: one of KDT_LIST_*, or -1 (the default)."""
    _check(_lib.kdt_set_large_k_list(tree.handle, int(placement)))


def kdt_large_k_list(tree: Tree, k: int) -> int:
    """The k-best list placement (KDT_LIST_*) that kdt_knn uses for this tree and k."""
    v = _I()
    _check(_lib.kdt_large_k_list(tree.handle, int(k), ctypes.byref(v)))
    return v.value


def kdt_tuned_params(tree: Tree, k: int):
    """(stage_levels, claim_steps, inline_depth, light_run) that kdt_knn uses for this tree and k."""
    a, b, c, d = _I(), _I(), _I(), _I()
    _check(_lib.kdt_tuned_params(tree.handle, k, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
    return a.value, b.value, c.value, d.value


def kdt_set_stage_levels(tree: Tree, levels: int) -> None:
    _check(_lib.kdt_set_stage_levels(tree.handle, int(levels)))


def kdt_autotune(tree: Tree, queries: torch.Tensor, k: int, flags: int = 0, stream=None):
    """Tune inline depth, claim steps and staging depth on these queries;
    returns (staging levels, ms); kdt_tuned_params gives all three."""
    Q = queries.shape[0]
    lv = _I()
    ms = _F()
    _check(_lib.kdt_autotune(tree.handle, _dev(queries, torch.float32, "queries", (Q, tree.D)), Q, k, flags,
                             ctypes.byref(lv), ctypes.byref(ms), _stream(stream)))
    return lv.value, ms.value


def kdt_tuning_save(path: str) -> None:
    _check(_lib.kdt_tuning_save(os.fsencode(path)))


def kdt_tuning_load(path: str) -> None:
    _check(_lib.kdt_tuning_load(os.fsencode(path)))


def kdt_debug_fail_allocs(n: int) -> None:
    """Make the library's next n device allocations fail with KDT_ENOMEM (tests)."""
    _check(_lib.kdt_debug_fail_allocs(n))


def kdt_debug_set_step_cap(tree: Tree, cap: int) -> None:
    """Lower the traversal step bound of a tree (0 restores 3N + 3; tests)."""
    _check(_lib.kdt_debug_set_step_cap(tree.handle, cap))


def kdt_profile_enable(tree: Tree, enable: bool = True) -> None:
    _check(_lib.kdt_profile_enable(tree.handle, int(bool(enable))))


def kdt_profile_read(tree: Tree):
    ms = _D()
    n = _I64()
    _check(_lib.kdt_profile_read(tree.handle, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


# ---------------------------------------------------------------- forests

def kdt_build_batched(points: torch.Tensor, offsets, stream=None) -> Forest:
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    D = points.shape[1]
    h = _P()
    _check(_lib.kdt_build_batched(_dev(points, torch.float32, "points"), ctypes.c_void_p(off.ctypes.data),
                                  len(off) - 1, D, _stream(stream), ctypes.byref(h)))
    return Forest(h, off, D)


def kdt_knn_batched(forest: Forest, queries: torch.Tensor, qoffsets, k: int, max_radius: float = math.inf,
                    flags: int = 0, out_ids=None, out_d2=None, stream=None):
    qoff = np.ascontiguousarray(qoffsets, dtype=np.int64)
    Q = int(qoff[-1])
    out_ids, out_d2 = _outputs(Q, k, out_ids, out_d2, queries.device)
    _check(_lib.kdt_knn_batched(forest.handle, _dev(queries, torch.float32, "queries", (Q, forest.D)),
                                ctypes.c_void_p(qoff.ctypes.data), k, float(max_radius), flags,
                                _dev(out_ids, torch.int32, "out_ids", (Q, k)),
                                _dev(out_d2, torch.float32, "out_d2", (Q, k)), _stream(stream)))
    return out_ids, out_d2


def kdt_knn_batched_visits(forest: Forest, queries: torch.Tensor, qoffsets, k: int, max_radius: float = math.inf,
                           flags: int = 0, stream=None) -> torch.Tensor:
    """Processed nodes of every query of the batched kNN (int32 [total queries])."""
    qoff = np.ascontiguousarray(qoffsets, dtype=np.int64)
    Q = int(qoff[-1])
    v = torch.empty(Q, dtype=torch.int32, device=queries.device)
    _check(_lib.kdt_knn_batched_visits(forest.handle, _dev(queries, torch.float32, "queries", (Q, forest.D)),
                                       ctypes.c_void_p(qoff.ctypes.data), k, float(max_radius), flags,
                                       _dev(v, torch.int32, "visits", (Q,)), _stream(stream)))
    return v


def kdt_forest_set_launch(forest: Forest, threads: int = 0, claim_steps: int = 0, inline_depth: int = 0,
                          light_run: int = 0) -> None:
    _check(_lib.kdt_forest_set_launch(forest.handle, threads, claim_steps, inline_depth, light_run))


def kdt_forest_autotune(forest: Forest, queries: torch.Tensor, query_offsets, k: int, max_radius: float = math.inf,
                        flags: int = 0, out_ids=None, out_d2=None, stream=None):
    """Tune inline depth, light run, block size and claim steps of the batched
    query; returns (threads, claim_steps, inline_depth, light_run, ms)."""
    qoff = np.ascontiguousarray(query_offsets, dtype=np.int64)
    Q = int(qoff[-1])
    out_ids, out_d2 = _outputs(Q, k, out_ids, out_d2, queries.device)
    th, cs, il, lr, ms = _I(), _I(), _I(), _I(), _F()
    _check(_lib.kdt_forest_autotune(forest.handle, _dev(queries, torch.float32, "queries", (Q, forest.D)),
                                    ctypes.c_void_p(qoff.ctypes.data), k, float(max_radius), flags,
                                    ctypes.c_void_p(out_ids.data_ptr()), ctypes.c_void_p(out_d2.data_ptr()),
                                    ctypes.byref(th), ctypes.byref(cs), ctypes.byref(il), ctypes.byref(lr),
                                    ctypes.byref(ms), _stream(stream)))
    return th.value, cs.value, il.value, lr.value, ms.value


def kdt_forest_export(forest: Forest, stream=None):
    total = int(forest.offsets[-1])
    coords = torch.empty((total, forest.D), dtype=torch.float32, device="cuda")
    ids = torch.empty(total, dtype=torch.int32, device="cuda")
    _check(_lib.kdt_forest_export(forest.handle, ctypes.c_void_p(coords.data_ptr()), ctypes.c_void_p(ids.data_ptr()),
                                  _stream(stream)))
    return coords, ids


def kdt_forest_free(forest: Forest) -> None:
    forest.free()


# ---------------------------------------------------------------- learned radius

def _need(name):
    fn = _OPTIONAL.get(name)
    if fn is None:
        raise KdtError(KDT_EINVAL, f"{name} is not exported by this libkdt.so")
    return fn


def kdt_radius_model_train(tree: Tree, train_queries: torch.Tensor, k: int, epochs: int = 0, batch: int = 0,
                           lr: float = 0.0, seed: int = 0, margin: float = 0.0, fallback_target: float = 0.0,
                           uniform_weights: bool = False, gate: int = KDT_GATE_AUTO, query_flags: int = 0,
                           stream=None) -> float:
    opts = TrainOpts(epochs, batch, lr, seed, margin, fallback_target, int(uniform_weights), int(gate),
                     int(query_flags))
    loss = _F()
    Qt = train_queries.shape[0]
    _check(_need("kdt_radius_model_train")(tree.handle, _dev(train_queries, torch.float32, "train_queries",
                                                             (Qt, tree.D)), Qt, k, ctypes.byref(opts),
                                           ctypes.byref(loss), _stream(stream)))
    return loss.value


def kdt_radius_model_get(tree: Tree):
    p = np.empty(MLP_PARAMS, dtype=np.float32)
    norm = np.empty(8, dtype=np.float32)
    m = _F()
    _check(_need("kdt_radius_model_get")(tree.handle, ctypes.c_void_p(p.ctypes.data), ctypes.c_void_p(norm.ctypes.data),
                                         ctypes.byref(m)))
    return p, norm, m.value


def kdt_radius_model_set(tree: Tree, params, norm, margin: float) -> None:
    p = np.ascontiguousarray(params, dtype=np.float32)
    n = np.ascontiguousarray(norm, dtype=np.float32)
    _check(_need("kdt_radius_model_set")(tree.handle, ctypes.c_void_p(p.ctypes.data), ctypes.c_void_p(n.ctypes.data),
                                         float(margin)))


def kdt_radius_model_save(tree: Tree, path: str) -> None:
    _check(_need("kdt_radius_model_save")(tree.handle, os.fsencode(path)))


def kdt_radius_model_load(tree: Tree, path: str) -> None:
    _check(_need("kdt_radius_model_load")(tree.handle, os.fsencode(path)))


def kdt_descent_features(tree: Tree, queries: torch.Tensor, stream=None) -> torch.Tensor:
    Q = queries.shape[0]
    f = torch.empty((Q, 4), dtype=torch.float32, device=queries.device)
    _check(_need("kdt_descent_features")(tree.handle, _dev(queries, torch.float32, "queries", (Q, tree.D)), Q,
                                         ctypes.c_void_p(f.data_ptr()), _stream(stream)))
    return f


def kdt_mlp_forward(params, x: torch.Tensor, stream=None) -> torch.Tensor:
    p = np.ascontiguousarray(params, dtype=np.float32)
    n = x.shape[0]
    y = torch.empty(n, dtype=torch.float32, device=x.device)
    _check(_need("kdt_mlp_forward")(ctypes.c_void_p(p.ctypes.data), _dev(x, torch.float32, "x", (n, 4)), n,
                                    ctypes.c_void_p(y.data_ptr()), _stream(stream)))
    return y


def kdt_mlp_loss_grad(params, x: torch.Tensor, label: torch.Tensor, stream=None):
    p = np.ascontiguousarray(params, dtype=np.float32)
    n = x.shape[0]
    g = np.empty(MLP_PARAMS, dtype=np.float32)
    loss = _F()
    _check(_need("kdt_mlp_loss_grad")(ctypes.c_void_p(p.ctypes.data), _dev(x, torch.float32, "x", (n, 4)),
                                      _dev(label, torch.float32, "label", (n,)), n, ctypes.byref(loss),
                                      ctypes.c_void_p(g.ctypes.data), _stream(stream)))
    return loss.value, g


def kdt_learned_stats(tree: Tree, stream=None):
    fb = _I64()
    ratio = _D()
    _check(_need("kdt_learned_stats")(tree.handle, ctypes.byref(fb), ctypes.byref(ratio), _stream(stream)))
    return fb.value, ratio.value


def kdt_learned_gated(tree: Tree, stream=None) -> int:
    """Queries of the last learned call that took the proposed radius."""
    n = _I64()
    _check(_need("kdt_learned_gated")(tree.handle, ctypes.byref(n), _stream(stream)))
    return n.value


def kdt_radius_model_gate(tree: Tree) -> int:
    g = _I()
    _check(_need("kdt_radius_model_gate")(tree.handle, ctypes.byref(g)))
    return g.value


def kdt_radius_model_set_gate(tree: Tree, gate: int) -> None:
    _check(_need("kdt_radius_model_set_gate")(tree.handle, int(gate)))


def kdt_l2_read_bandwidth(nbytes: int = 32 << 20, reps: int = 200, stream=None) -> float:
    """L2 read bandwidth of the current GPU in GB/s (the library's own probe kernel)."""
    v = _D()
    _check(_lib.kdt_l2_read_bandwidth(int(nbytes), int(reps), ctypes.byref(v), _stream(stream)))
    return v.value
