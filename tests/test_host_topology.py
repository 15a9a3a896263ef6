"""The CUDA builder's closed-form tree topology, checked on the CPU.

The builder never walks the tree: it maps level-order node indices to in-order
positions and back, and finds subtree ends, by closed forms on (n, t)
(`Topo` in the library's internal header; the complete left-balanced tree of
Sec. 3, children 2t+1 and 2t+2).  Those forms are host/device functions, so a
small host-only probe compiled with nvcc prints them here, and this test
compares them with a plain enumeration (every n up to 600) and, for sizes up
to 2^30 - 1 that no enumeration reaches, with subtree sizes counted level by
level.  The float sort key is checked against float order.
"""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROBE_SRC = os.path.join(ROOT, "tests", "host", "topo_probe.cu")

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="needs nvcc")


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path_factory.mktemp("probe") / "topo_probe")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a", "-o", exe,
                    PROBE_SRC], check=True, capture_output=True)

    def run(lines):
        r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return r.stdout.split("\n")[: len(lines)]

    return run


def _enumerate(n):
    """In-order sequence of a level-order complete tree of n nodes, by walking it."""
    order, stack, t = [], [], 0
    while stack or t < n:
        while t < n:
            stack.append(t)
            t = 2 * t + 1
        t = stack.pop()
        order.append(t)
        t = 2 * t + 2
    return order


def _size(i, n):
    """Nodes of the subtree of i: on each level below i it holds the index
    range [(i+1)2^m - 1, (i+2)2^m - 2], cut at n."""
    s, m = 0, 0
    while (i + 1) * (1 << m) - 1 < n:
        lo = (i + 1) * (1 << m) - 1
        hi = min((i + 2) * (1 << m) - 2, n - 1)
        s += hi - lo + 1
        m += 1
    return s


def _inorder_by_sizes(t, n):
    """In-order position of t: its left subtree, plus, for every ancestor whose
    right subtree holds t, that ancestor's left subtree and the ancestor."""
    pos = _size(2 * t + 1, n) if 2 * t + 1 < n else 0
    u = t
    while u > 0:
        parent = (u - 1) // 2
        if u == 2 * parent + 2:
            pos += _size(2 * parent + 1, n) + 1
        u = parent
    return pos


def _node_at_by_sizes(p, n):
    u = 0
    while True:
        left = _size(2 * u + 1, n) if 2 * u + 1 < n else 0
        if p == left:
            return u
        if p < left:
            u = 2 * u + 1
        else:
            p -= left + 1
            u = 2 * u + 2


def _ends(t, n):
    lo = t
    while 2 * lo + 1 < n:
        lo = 2 * lo + 1
    hi = t
    while 2 * hi + 2 < n:
        hi = 2 * hi + 2
    # a right spine can end at a node whose only child is a left one
    return lo, hi


def test_topology_maps_every_small_tree(probe):
    cases, want = [], []
    for n in range(1, 601):
        order = _enumerate(n)
        pos = {t: p for p, t in enumerate(order)}
        for t in range(n):
            lo, hi = _ends(t, n)
            cases.append(f"t {n} {t}")
            want.append(f"{(t + 1).bit_length() - 1} {pos[t]} {order[t]} {lo} {hi}")
    got = probe(cases)
    bad = [(c, g, w) for c, g, w in zip(cases, got, want) if g != w]
    assert not bad, bad[:5]


def test_topology_maps_up_to_the_size_limit(probe):
    g = np.random.default_rng(3)
    sizes = [2 ** 30 - 1, 2 ** 30 - 2, 2 ** 29, 2 ** 29 + 1, 2 ** 24, 2 ** 24 + 12345, 155500788,
             int(g.integers(2 ** 20, 2 ** 30))]
    cases, want = [], []
    for n in sizes:
        ts = {0, 1, 2, n - 1, n - 2, n // 2, (n - 1) // 2, (n - 2) // 2}
        ts |= {int(x) for x in g.integers(0, n, 200)}
        for t in sorted(x for x in ts if 0 <= x < n):
            lo, hi = _ends(t, n)
            cases.append(f"t {n} {t}")
            want.append(f"{(t + 1).bit_length() - 1} {_inorder_by_sizes(t, n)} {_node_at_by_sizes(t, n)} {lo} {hi}")
    got = probe(cases)
    bad = [(c, g_, w) for c, g_, w in zip(cases, got, want) if g_ != w]
    assert not bad, bad[:5]


def test_float_key_preserves_float_order(probe):
    g = np.random.default_rng(4)
    vals = np.concatenate([
        np.array([0.0, -0.0, 1.0, -1.0, 1e-45, -1e-45, 1.17549435e-38, -1.17549435e-38, 3.4028235e38,
                  -3.4028235e38, 0.5, -0.5], dtype=np.float32),
        (g.standard_normal(400) * 10.0 ** g.integers(-30, 30, 400)).astype(np.float32),
        g.integers(-3, 4, 50).astype(np.float32),
    ])
    vals = vals[np.isfinite(vals)]
    bits = [struct.unpack("<I", struct.pack("<f", float(v)))[0] for v in vals]
    keys = np.array([int(x) for x in probe([f"k {b:08x}" for b in bits])], dtype=np.int64)
    order = np.argsort(vals, kind="stable")
    sv, sk = vals[order], keys[order]
    # keys ascend with the floats, and are equal exactly where the floats are
    # (-0 and +0 share a key)
    assert np.all((sv[1:] > sv[:-1]) == (sk[1:] > sk[:-1]))
    assert np.all((sv[1:] == sv[:-1]) == (sk[1:] == sk[:-1]))
