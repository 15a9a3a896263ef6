"""GPU parity of the traversal ablations: the stack-free machine as stated
(one node per step), the swapped order (node after its close subtree) and a
stack-based traversal.  Results are bit-identical to kdt_knn's and to brute
force; processed-node counts equal the oracle's traversal in the same order
(root first for the plain and stack-based kernels, close first for the swap)."""
import math

import numpy as np
import pytest

import oracle
from paper_2210_12859_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CLOSE_FIRST = 2


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


VARIANTS = ["PLAIN_STEP", "CLOSE_FIRST", "STACK"]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("D,N,widest", [(1, 3000, 0), (2, 5000, 0), (3, 20000, 0), (4, 8000, 0), (3, 20000, 1)])
def test_ablation_equals_plain_and_oracle_visits(kdt, variant, D, N, widest):
    g = np.random.default_rng(D * 7 + N + widest)
    pts = synth.uniform(N, D, seed=D + N)
    if N == 3000:
        pts = g.integers(0, 50, size=(N, D)).astype(np.float32)  # duplicates and ties
    qs = (g.random((300, D)) * 1.2 - 0.1).astype(np.float32)
    flag = getattr(kdt, "KDT_" + variant)
    tree = kdt.kdt_build(cu(pts), opts=kdt.KDT_BUILD_WIDEST if widest else 0)
    if widest:
        pid, dims = oracle.build_widest(pts)
    else:
        pid, dims = oracle.build(pts), None
    order = CLOSE_FIRST if variant == "CLOSE_FIRST" else True
    for k, r in ((1, math.inf), (5, math.inf), (8, 0.05), (16, math.inf)):
        for morton in (0, kdt.KDT_MORTON):
            pi, pd = kdt.kdt_knn(tree, cu(qs), k, r, flags=morton)
            ai, ad = kdt.kdt_knn(tree, cu(qs), k, r, flags=flag | morton)
            kdt.kdt_status(tree)
            assert torch.equal(pi, ai) and torch.equal(pd.view(torch.int32), ad.view(torch.int32)), (k, r)
        v = kdt.kdt_knn_visits(tree, cu(qs), k, r, flags=flag).cpu().numpy()
        if dims is None:
            _, _, want_v = oracle.knn_tree(pts, pid, qs, k, r, ordered=order)
        else:
            _, _, want_v = oracle.knn_tree_dims(pts, pid, dims, qs, k, r, ordered=order)
        assert np.array_equal(v, want_v), (k, r)
    wi, wd = oracle.knn_brute(pts, qs, 8, 0.05)
    ai, ad = kdt.kdt_knn(tree, cu(qs), 8, 0.05, flags=flag)
    assert np.array_equal(ai.cpu().numpy(), wi) and np.array_equal(bits(ad.cpu().numpy()), bits(wd))


def test_stack_and_plain_step_visit_the_same_nodes(kdt):
    """Sec. 3.1's recursion and the stack-free machine process the same nodes:
    the explicit-stack kernel and the one-node-per-step kernel agree per query,
    and both agree with the production kernel's visit counts."""
    mix = synth.gmm_mixture(16, 3, 0.02, 3)
    pts = synth.gmm_sample(mix, 1 << 17, 4)
    qs = synth.gmm_queries(mix, 4096, 0.1, 5)
    tree = kdt.kdt_build(cu(pts))
    for k in (1, 8, 16):
        a = kdt.kdt_knn_visits(tree, cu(qs), k, flags=kdt.KDT_STACK)
        b = kdt.kdt_knn_visits(tree, cu(qs), k, flags=kdt.KDT_PLAIN_STEP)
        c = kdt.kdt_knn_visits(tree, cu(qs), k)
        assert torch.equal(a, b) and torch.equal(b, c)


def test_ablation_rejects_bad_combinations(kdt):
    pts = synth.uniform(1000, 3, seed=1)
    tree = kdt.kdt_build(cu(pts))
    q = cu(pts[:8])
    bad = [(8, kdt.KDT_STACK | kdt.KDT_CLOSE_FIRST), (8, kdt.KDT_STACK | kdt.KDT_UNORDERED),
           (8, kdt.KDT_PLAIN_STEP | kdt.KDT_LEARNED), (17, kdt.KDT_STACK)]
    for k, f in bad:
        with pytest.raises(kdt.KdtError):
            kdt.kdt_knn(tree, q, k, flags=f)
    t6 = kdt.kdt_build(cu(synth.uniform(1000, 6, seed=2)))
    with pytest.raises(kdt.KdtError):
        kdt.kdt_knn(t6, cu(synth.uniform(4, 6, seed=3)), 4, flags=kdt.KDT_CLOSE_FIRST)
