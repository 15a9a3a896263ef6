"""Launch tuning never changes a result: every staging depth, claim interval
and inline depth gives the same bits and the same processed-node counts; the
autotuner picks one of its candidates and its choice survives a save / load
round trip."""
import json
import os

import numpy as np
import pytest

from paper_2210_12859_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kdt():
    from paper_2210_12859_gb300 import build

    build.build_library()
    from paper_2210_12859_gb300 import kdt as k

    return k


def test_staging_depths_identical(kdt):
    pts, qs = synth.uniform_small(1 << 15, 20000)
    tree = kdt.kdt_build(torch.from_numpy(pts).cuda())
    dq = torch.from_numpy(qs).cuda()
    ref = None
    for lv in (0, 1, 5, 11, 13, -1):
        kdt.kdt_set_stage_levels(tree, lv)
        for flags in (kdt.KDT_MORTON, kdt.KDT_UNORDERED):
            r = kdt.kdt_knn(tree, dq, 8, flags=flags)
            if ref is None:
                ref = r
            assert torch.equal(r[0], ref[0]) and torch.equal(r[1], ref[1])
    with pytest.raises(kdt.KdtError):
        kdt.kdt_set_stage_levels(tree, 17)


@pytest.mark.parametrize("k", [1, 8, 32])
def test_claim_steps_and_inline_depth_identical(kdt, k):
    mix = synth.gmm_mixture(16, 3, 0.02, 4)
    pts = synth.gmm_sample(mix, 1 << 16, 5)
    qs = synth.gmm_queries(mix, 20000, 0.1, 6)
    tree = kdt.kdt_build(torch.from_numpy(pts).cuda())
    dq = torch.from_numpy(qs).cuda()
    ref = kdt.kdt_knn(tree, dq, k, flags=kdt.KDT_MORTON)
    ref_v = kdt.kdt_knn_visits(tree, dq, k)
    for depth, lr in ((0, 1), (1, 4), (2, 1), (2, 8), (1, 64), (3, 1), (3, 4), (4, 1)):
        for cs in (1, 7, 16, 64, 256):
            kdt.kdt_set_inline_depth(tree, depth)
            kdt.kdt_set_claim_steps(tree, cs)
            kdt.kdt_set_light_run(tree, lr)
            assert kdt.kdt_tuned_params(tree, k)[1:] == (cs, depth, lr)
            for flags in (kdt.KDT_MORTON, kdt.KDT_UNORDERED, 0):
                r = kdt.kdt_knn(tree, dq, k, flags=flags)
                assert torch.equal(r[0], ref[0]) and torch.equal(r[1], ref[1]), (depth, cs, flags)
            assert torch.equal(kdt.kdt_knn_visits(tree, dq, k), ref_v)
    for bad in ((kdt.kdt_set_inline_depth, 5), (kdt.kdt_set_claim_steps, 0), (kdt.kdt_set_claim_steps, 257),
                (kdt.kdt_set_light_run, 0), (kdt.kdt_set_light_run, 65)):
        with pytest.raises(kdt.KdtError):
            bad[0](tree, bad[1])
    kdt.kdt_set_inline_depth(tree, -1)
    kdt.kdt_set_claim_steps(tree, -1)
    kdt.kdt_set_light_run(tree, -1)
    assert kdt.kdt_tuned_params(tree, 1) == (0, 32, 2, 1)
    assert kdt.kdt_tuned_params(tree, 8) == (0, 64, 2, 1)


def test_autotune_and_tuning_file(kdt, tmp_path):
    pts, qs = synth.gmm_large(1 << 18, 1 << 16)
    tree = kdt.kdt_build(torch.from_numpy(pts).cuda())
    dq = torch.from_numpy(qs).cuda()
    lv, ms = kdt.kdt_autotune(tree, dq, 8, kdt.KDT_MORTON)
    assert lv in (0, 4, 6, 8) and ms > 0
    tlv, cs, depth, lr = kdt.kdt_tuned_params(tree, 8)
    assert tlv == lv and cs in (16, 32, 64, 128) and depth in (0, 1, 2, 3, 4) and lr in (1, 4, 8)
    path = os.path.join(tmp_path, "tuning.json")
    kdt.kdt_tuning_save(path)
    rows = json.load(open(path))
    assert any(r["D"] == 3 and r["log2n"] == 18 and r["stage_levels"] == lv and r["claim_steps"] == cs and
               r["inline_depth"] == depth and r["light_run"] == lr for r in rows)
    kdt.kdt_tuning_load(path)
    a = kdt.kdt_knn(tree, dq, 8, flags=kdt.KDT_MORTON)
    kdt.kdt_set_stage_levels(tree, 0)
    b = kdt.kdt_knn(tree, dq, 8, flags=kdt.KDT_MORTON)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    open(path, "w").write('[\n  {"gpu": "x", "D": 3, "k_bucket": 3, "log2n": 18, "stage_levels": 99}\n]\n')
    with pytest.raises(kdt.KdtError):
        kdt.kdt_tuning_load(path)
    open(path, "w").write('[\n  {"gpu": "x", "D": 3, "k_bucket": 3, "log2n": 18, "stage_levels": 0, '
                          '"claim_steps": 64, "inline_depth": 5}\n]\n')
    with pytest.raises(kdt.KdtError):
        kdt.kdt_tuning_load(path)
    # rows written before the claim / inline fields existed still load
    open(path, "w").write('[\n  {"gpu": "x", "D": 3, "k_bucket": 3, "log2n": 18, "stage_levels": 4}\n]\n')
    kdt.kdt_tuning_load(path)


@pytest.mark.parametrize("N,D,widest", [(1 << 16, 3, False), (50001, 3, False), (9, 3, False), (23, 2, False),
                                        (47, 3, False), (24, 3, True), (1 << 17, 3, False), (98303, 2, False),
                                        (100003, 4, False), (40000, 8, False), (70001, 3, True), (131071, 1, False)])
def test_deep_inline_depths_identical(kdt, N, D, widest):
    """The depth-3 and depth-4 steps (a node and the whole subtree below it, as
    depth-2 blocks, in one step) on complete and ragged last levels, every node
    layout and a stored split dimension: the same results and processed nodes
    as depth 2, both orders."""
    g = np.random.default_rng(N + D)
    pts = g.random((N, D), dtype=np.float32)
    qs = g.random((6000, D), dtype=np.float32) * 1.2 - 0.1
    tree = kdt.kdt_build(torch.from_numpy(pts).cuda(), opts=kdt.KDT_BUILD_WIDEST if widest else 0)
    dq = torch.from_numpy(qs).cuda()
    for k in (1, 8, 16, 32):
        for flags in (kdt.KDT_MORTON, kdt.KDT_UNORDERED):
            kdt.kdt_set_inline_depth(tree, 2)
            want = kdt.kdt_knn(tree, dq, k, flags=flags)
            want_v = kdt.kdt_knn_visits(tree, dq, k, flags=flags)
            for depth in (3, 4):
                kdt.kdt_set_inline_depth(tree, depth)
                got = kdt.kdt_knn(tree, dq, k, flags=flags)
                got_v = kdt.kdt_knn_visits(tree, dq, k, flags=flags)
                assert torch.equal(got[0], want[0]) and torch.equal(got[1].view(torch.int32),
                                                                    want[1].view(torch.int32)), (depth, k, flags)
                assert torch.equal(got_v, want_v), (depth, k, flags)
    kdt.kdt_status(tree)


@pytest.mark.parametrize("N,D", [(1 << 16, 3), (50001, 3), (30000, 4), (70, 3)])
def test_large_k_list_placements_identical(kdt, N, D):
    """k > 16: the shared-memory heap, the same heap in global scratch, and the
    lists spread over 4 or 8 lanes with shuffle insertion give the same ids,
    distance bits and processed nodes, both orders, with and without a radius,
    for k that fill the 4- and 8-lane blocks partly and fully."""
    g = np.random.default_rng(N)
    pts = g.random((N, D), dtype=np.float32)
    qs = (g.random((5000, D)) * 1.2 - 0.1).astype(np.float32)
    tree = kdt.kdt_build(torch.from_numpy(pts).cuda())
    dq = torch.from_numpy(qs).cuda()
    for k in (17, 32, 33, 64):
        for flags, r in ((kdt.KDT_MORTON, float("inf")), (kdt.KDT_UNORDERED, float("inf")), (0, 0.08)):
            kdt.kdt_set_large_k_list(tree, kdt.KDT_LIST_SHARED)
            want = kdt.kdt_knn(tree, dq, k, r, flags=flags)
            want_v = kdt.kdt_knn_visits(tree, dq, k, r, flags=flags)
            for placement in (kdt.KDT_LIST_GLOBAL, kdt.KDT_LIST_GROUP4, kdt.KDT_LIST_GROUP8):
                kdt.kdt_set_large_k_list(tree, placement)
                for depth in (2, 3):
                    kdt.kdt_set_inline_depth(tree, depth)
                    got = kdt.kdt_knn(tree, dq, k, r, flags=flags)
                    assert torch.equal(got[0], want[0]), (k, placement, depth)
                    assert torch.equal(got[1].view(torch.int32), want[1].view(torch.int32)), (k, placement, depth)
                    assert torch.equal(kdt.kdt_knn_visits(tree, dq, k, r, flags=flags), want_v), (k, placement)
                kdt.kdt_set_inline_depth(tree, -1)
    with pytest.raises(kdt.KdtError):
        kdt.kdt_set_large_k_list(tree, 9)
    kdt.kdt_set_large_k_list(tree, -1)
    kdt.kdt_status(tree)
