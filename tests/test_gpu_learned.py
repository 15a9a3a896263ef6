"""GPU parity of the learned radius proposal.

The proposal must never change a result: learned == plain, bit for bit.  Its
parts are checked against the oracle: descent features (exact coordinates,
log of the oracle's leaf distance within the rounding of logf), MLP forward
and gradients (FP64 oracle on the same BF16-rounded weights, FP32
accumulation tolerance).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2210_12859_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = 64 * 4 + 64 + 64 * 64 + 64 + 64 + 1
H = 64


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


def weight_mask():
    m = np.zeros(P, dtype=bool)
    m[: 4 * H] = True                       # W1
    m[5 * H: 5 * H + H * H] = True          # W2
    m[6 * H + H * H: 7 * H + H * H] = True  # w3
    return m


def rounded(params):
    p = np.asarray(params, dtype=np.float32).copy()
    m = weight_mask()
    p[m] = [oracle.round_bf16(float(v)) for v in p[m]]
    return p.astype(np.float64)


def random_params(seed, scale=0.3):
    g = np.random.default_rng(seed)
    return (g.standard_normal(P) * scale).astype(np.float32)


@pytest.fixture(scope="module")
def surface(kdt):
    """Surface data (spheres and tori), N = 2^18, for the learned path."""
    pts, qs = synth.surface_set(1 << 18, 3 << 14)
    tree = kdt.kdt_build(cu(pts))
    return pts, qs, tree


def test_descent_features_match_oracle(kdt, surface):
    pts, qs, tree = surface
    sub = qs[:4000]
    f = kdt.kdt_descent_features(tree, cu(sub)).cpu().numpy()
    assert np.array_equal(bits(f[:, :3]), bits(sub))
    _, node_ids = kdt.kdt_tree_export(tree)
    d2 = oracle.descent_leaf_d2(pts, node_ids.cpu().numpy(), sub)
    want = np.log(np.maximum(d2, np.float32(1e-30)).astype(np.float64))
    # same d2 bits on both sides; the device's logf (documented error 1 ulp)
    # against FP64 log: allow about 30 FP32 ulps of the largest feature
    assert np.allclose(f[:, 3], want, rtol=0, atol=4e-6 * np.maximum(1.0, np.abs(want)).max())


def test_descent_features_stored_dims_match_oracle(kdt, surface):
    """Features on a tree that stores each node's widest dimension: the
    device descent reads the dimension kept in the node's id word; the
    oracle descends its own widest-split tree with its recorded dimensions."""
    pts, qs, _ = surface
    sub = qs[:4000]
    pid, dims = oracle.build_widest(pts)
    tree = kdt.kdt_build(cu(pts), opts=kdt.KDT_BUILD_WIDEST)
    try:
        f = kdt.kdt_descent_features(tree, cu(sub)).cpu().numpy()
        assert np.array_equal(kdt.kdt_tree_split_dims(tree).cpu().numpy(), dims)
    finally:
        tree.free()
    assert np.array_equal(bits(f[:, :3]), bits(sub))
    d2 = oracle.descent_leaf_d2(pts, pid, sub, node_dim=dims)
    # the stored dimensions change the descent on this data
    assert not np.array_equal(d2, oracle.descent_leaf_d2(pts, oracle.build(pts), sub))
    want = np.log(np.maximum(d2, np.float32(1e-30)).astype(np.float64))
    assert np.allclose(f[:, 3], want, rtol=0, atol=4e-6 * np.maximum(1.0, np.abs(want)).max())


def test_mlp_forward_matches_oracle(kdt):
    """The inference forward (hidden layer on the tensor cores, BF16 operands,
    FP32 accumulation) against the oracle's FP64 model with the same
    bfloat16-valued weights, within the oracle's per-sample bound for any
    BF16-in / FP32-accumulate evaluation (the bfloat16 rounding of the 64
    hidden activations, unit roundoff 2^-8, carried through both layers, plus
    an FP32 allowance of 2^-23 per operation); 5000 samples = 40 tiles of 128
    with a ragged last tile."""
    p = random_params(1)
    g = np.random.default_rng(2)
    x = g.standard_normal((5000, 4)).astype(np.float32)
    y = kdt.kdt_mlp_forward(p, cu(x)).cpu().numpy().astype(np.float64)
    want, bound = oracle.mlp_forward_bound(rounded(p), H, x.astype(np.float64))
    err = np.abs(y - want)
    assert np.all(err <= bound), float(np.max(err / bound))
    # the tensor-core result is not the FP64 model's: the rounding shows
    assert err.max() > 0


@pytest.mark.parametrize("n", [1000, 128, 77])
def test_mlp_gradients_match_oracle(kdt, n):
    """Loss and gradient of the tensor-core training step (BF16 operands in the
    64 x 64 contractions, FP32 accumulation) against the oracle's FP64 loss
    and gradient with the same bfloat16 weights, each parameter within the
    oracle's bound for any BF16-in / FP32 evaluation (the bfloat16 rounding of
    the hidden activations and of the back-propagated gradient, ReLUs within
    their error of 0 admitted either way, 2^-23 per FP32 operation); several
    128-sample tiles with a ragged last one, one full tile, one partial tile."""
    p = random_params(3)
    g = np.random.default_rng(4)
    x = g.standard_normal((n, 4)).astype(np.float32)
    lab = g.standard_normal(n).astype(np.float32)
    loss, grad = kdt.kdt_mlp_loss_grad(p, cu(x), cu(lab))
    wl, wg, bound, lbound = oracle.mlp_loss_grad_bound(rounded(p), H, x.astype(np.float64), lab.astype(np.float64))
    err = np.abs(np.asarray(grad, dtype=np.float64) - wg)
    assert np.all(err <= bound), float(np.max(err / np.maximum(bound, 1e-300)))
    assert abs(loss - wl) <= lbound + 1e-7 * abs(wl)  # + the final FP32 division by n
    # the rounding shows: the tensor-core gradient is not the FP64 one
    assert err.max() > 0


@pytest.fixture(scope="module")
def trained(kdt, surface):
    pts, qs, tree = surface
    train = cu(qs[: 1 << 15])
    # every query takes the proposal: these tests look at the proposal itself
    loss = kdt.kdt_radius_model_train(tree, train, 8, epochs=10, batch=1024, seed=7, gate=kdt.KDT_GATE_ALL)
    return loss


@pytest.mark.parametrize("uniform_weights", [False, True])
def test_training_fits_radii(kdt, uniform_weights):
    """On clustered data with 10% far queries the k-th neighbour radius spans
    orders of magnitude; the trained model must explain most of its variance.
    Unweighted training calibrates the margin for 2% re-runs by count; the
    default cost-weighted training for re-runs worth about 2% of the plain
    work, so the total work stays close to the plain method's."""
    mix = synth.gmm_mixture(64, 3, 0.01, 9)
    pts = synth.gmm_sample(mix, 1 << 18, 10)
    q = synth.gmm_queries(mix, 1 << 15, 0.1, 11)
    tree = kdt.kdt_build(cu(pts))
    loss = kdt.kdt_radius_model_train(tree, cu(q), 8, epochs=10, batch=1024, seed=3,
                                      uniform_weights=uniform_weights)
    _, d2 = kdt.kdt_knn(tree, cu(q), 8)
    lab = 0.5 * np.log(np.maximum(d2.cpu().numpy()[:, -1].astype(np.float64), 1e-30))
    assert loss < 0.25 * lab.var(), (loss, lab.var())
    qe = cu(synth.gmm_queries(mix, 1 << 14, 0.1, 12))
    a = kdt.kdt_knn(tree, qe, 8)
    b = kdt.kdt_knn(tree, qe, 8, flags=kdt.KDT_LEARNED)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    fb, ratio = kdt.kdt_learned_stats(tree)
    _, _, margin = kdt.kdt_radius_model_get(tree)
    assert 1.0 < margin < 16.0
    if uniform_weights:
        assert fb < 0.06 * qe.shape[0], fb
    else:
        assert fb < 0.2 * qe.shape[0], fb
        plain = kdt.kdt_knn_visits(tree, qe, 8).double().sum().item()
        learned = kdt.kdt_knn_visits(tree, qe, 8, flags=kdt.KDT_LEARNED).double().sum().item()
        assert learned < 1.05 * plain, (learned, plain)


def test_fixed_margin_as_configured(kdt, surface):
    """The learned-radius configuration fixes the cull radius at 1.25 x the
    prediction: a margin given to the training is kept as is (no
    calibration), and the results stay those of the plain method."""
    pts, qs, _ = surface
    tree = kdt.kdt_build(cu(pts))  # its own tree: the module's tree keeps its model
    kdt.kdt_radius_model_train(tree, cu(qs[: 1 << 14]), 8, epochs=4, batch=1024, seed=5, margin=1.25)
    _, _, margin = kdt.kdt_radius_model_get(tree)
    assert margin == 1.25
    q = cu(qs[1 << 15:])
    for k in (8, 32):
        pi, pd = kdt.kdt_knn(tree, q, k, flags=kdt.KDT_MORTON)
        li, ld = kdt.kdt_knn(tree, q, k, flags=kdt.KDT_MORTON | kdt.KDT_LEARNED)
        assert torch.equal(pi, li) and torch.equal(pd.view(torch.int32), ld.view(torch.int32))
    kdt.kdt_status(tree)


@pytest.mark.parametrize("k", [8, 32])
@pytest.mark.parametrize("flags_name", ["MORTON", "ORDERED"])
def test_learned_equals_plain(kdt, surface, trained, k, flags_name):
    pts, qs, tree = surface
    flags = getattr(kdt, "KDT_" + flags_name)
    q = cu(qs[1 << 15:])
    pi, pd = kdt.kdt_knn(tree, q, k, flags=flags)
    li, ld = kdt.kdt_knn(tree, q, k, flags=flags | kdt.KDT_LEARNED)
    assert torch.equal(pi, li)
    assert torch.equal(pd.view(torch.int32), ld.view(torch.int32))
    fb, ratio = kdt.kdt_learned_stats(tree)
    assert 0 <= fb < q.shape[0]
    if k == 8:
        assert 1.0 <= ratio < 3.0
    kdt.kdt_status(tree)


def test_learned_bounded_radius_equals_plain(kdt, surface, trained):
    pts, qs, tree = surface
    q = cu(qs[1 << 15:])
    for r in (0.002, 0.01, 1.0):
        pi, pd = kdt.kdt_knn(tree, q, 8, r)
        li, ld = kdt.kdt_knn(tree, q, 8, r, flags=kdt.KDT_LEARNED)
        assert torch.equal(pi, li) and torch.equal(pd.view(torch.int32), ld.view(torch.int32))
    # and against the oracle on a sample
    sample = np.arange(0, q.shape[0], 97)
    wi, wd = oracle.knn_brute(pts, qs[1 << 15:][sample], 8, 0.01)
    li, ld = kdt.kdt_knn(tree, q, 8, 0.01, flags=kdt.KDT_LEARNED)
    assert np.array_equal(li.cpu().numpy()[sample], wi)
    assert np.array_equal(bits(ld.cpu().numpy()[sample]), bits(wd))


def test_learned_visits_fewer_nodes(kdt, surface, trained):
    """What the trained network gains: fewer processed nodes per query than
    the plain ordered traversal, at identical results."""
    pts, qs, tree = surface
    q = cu(qs[1 << 15:])
    plain = kdt.kdt_knn_visits(tree, q, 8).double().mean().item()
    learned = kdt.kdt_knn_visits(tree, q, 8, flags=kdt.KDT_LEARNED).double().mean().item()
    assert learned < plain, (learned, plain)


def test_model_save_load_roundtrip(kdt, surface, trained, tmp_path):
    pts, qs, tree = surface
    path = os.path.join(tmp_path, "radius.bin")
    kdt.kdt_radius_model_save(tree, path)
    p1, n1, m1 = kdt.kdt_radius_model_get(tree)
    other = kdt.kdt_build(cu(pts))
    kdt.kdt_radius_model_load(other, path)
    p2, n2, m2 = kdt.kdt_radius_model_get(other)
    assert np.array_equal(p1, p2) and np.array_equal(n1, n2) and m1 == m2
    assert kdt.kdt_radius_model_gate(other) == kdt.kdt_radius_model_gate(tree)
    kdt.kdt_radius_model_set_gate(other, kdt.KDT_GATE_FAR)
    kdt.kdt_radius_model_save(other, path)
    third = kdt.kdt_build(cu(pts))
    kdt.kdt_radius_model_load(third, path)
    assert kdt.kdt_radius_model_gate(third) == kdt.KDT_GATE_FAR
    q = cu(qs[1 << 15: (1 << 15) + 5000])
    a = kdt.kdt_knn(tree, q, 8, flags=kdt.KDT_LEARNED)
    b = kdt.kdt_knn(other, q, 8, flags=kdt.KDT_LEARNED)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    with open(path, "r+b") as f:
        f.write(b"XXXX")
    with pytest.raises(kdt.KdtError) as e:
        kdt.kdt_radius_model_load(other, path)
    assert e.value.code == kdt.KDT_EIO


def test_learned_rejects_untrained_and_high_dim(kdt):
    pts = synth.uniform(1000, 4, seed=1)
    t = kdt.kdt_build(cu(pts))
    with pytest.raises(kdt.KdtError):
        kdt.kdt_radius_model_train(t, cu(pts), 8)
    t3 = kdt.kdt_build(cu(pts[:, :3].copy()))
    with pytest.raises(kdt.KdtError) as e:
        kdt.kdt_knn(t3, cu(pts[:10, :3].copy()), 8, flags=kdt.KDT_LEARNED)
    assert e.value.code == kdt.KDT_ENOMODEL


@pytest.fixture(scope="module")
def clustered(kdt):
    """Clustered points with 10 % of the queries between the clusters, and a
    model trained on them (every query gated)."""
    mix = synth.gmm_mixture(64, 3, 0.01, 21)
    pts = synth.gmm_sample(mix, 1 << 18, 22)
    train = synth.gmm_queries(mix, 1 << 15, 0.1, 23)
    qs = synth.gmm_queries(mix, 30001, 0.1, 24)
    tree = kdt.kdt_build(cu(pts))
    kdt.kdt_radius_model_train(tree, cu(train), 8, epochs=8, batch=1024, seed=9, gate=kdt.KDT_GATE_ALL)
    return pts, qs, tree


@pytest.mark.parametrize("flags_name", ["MORTON", "MORTON|COST_ORDER", "ORDERED", "UNORDERED"])
def test_every_gate_equals_plain(kdt, clustered, flags_name):
    """All queries, the far ones only, or none take the proposal: the same
    results and, with no query gated, the plain method's processed nodes.  The
    far gate takes the queries whose greedy descent ends far outside the data,
    about the 10 % drawn between the clusters."""
    pts, qs, tree = clustered
    flags = 0
    for n in flags_name.split("|"):
        flags |= getattr(kdt, "KDT_" + n)
    q = cu(qs)
    Q = qs.shape[0]
    pi, pd = kdt.kdt_knn(tree, q, 8, flags=flags)
    pv = kdt.kdt_knn_visits(tree, q, 8, flags=flags)
    for gate in (kdt.KDT_GATE_ALL, kdt.KDT_GATE_FAR, kdt.KDT_GATE_NONE):
        kdt.kdt_radius_model_set_gate(tree, gate)
        assert kdt.kdt_radius_model_gate(tree) == gate
        li, ld = kdt.kdt_knn(tree, q, 8, flags=flags | kdt.KDT_LEARNED)
        assert torch.equal(pi, li) and torch.equal(pd.view(torch.int32), ld.view(torch.int32)), gate
        gated = kdt.kdt_learned_gated(tree)
        fb, ratio = kdt.kdt_learned_stats(tree)
        assert 0 <= fb <= gated
        if gate == kdt.KDT_GATE_ALL:
            assert gated == Q
        elif gate == kdt.KDT_GATE_FAR:
            assert 0.05 * Q < gated < 0.15 * Q, gated
            assert ratio >= 1.0
        else:
            assert gated == 0 and fb == 0
            assert torch.equal(kdt.kdt_knn_visits(tree, q, 8, flags=flags | kdt.KDT_LEARNED), pv)
    kdt.kdt_radius_model_set_gate(tree, kdt.KDT_GATE_ALL)
    with pytest.raises(kdt.KdtError):
        kdt.kdt_radius_model_set_gate(tree, 7)
    kdt.kdt_status(tree)


def test_automatic_gate(kdt, clustered):
    """Training with the default gate times the plain and the gated forms on
    the training queries and keeps one of them; the results stay the plain
    method's."""
    pts, qs, _ = clustered
    mix = synth.gmm_mixture(64, 3, 0.01, 21)
    tree = kdt.kdt_build(cu(pts))
    kdt.kdt_radius_model_train(tree, cu(synth.gmm_queries(mix, 1 << 15, 0.1, 25)), 8, epochs=4, batch=1024, seed=2)
    assert kdt.kdt_radius_model_gate(tree) in (kdt.KDT_GATE_ALL, kdt.KDT_GATE_FAR, kdt.KDT_GATE_NONE)
    q = cu(qs)
    flags = kdt.KDT_MORTON | kdt.KDT_COST_ORDER
    pi, pd = kdt.kdt_knn(tree, q, 8, flags=flags)
    li, ld = kdt.kdt_knn(tree, q, 8, flags=flags | kdt.KDT_LEARNED)
    assert torch.equal(pi, li) and torch.equal(pd.view(torch.int32), ld.view(torch.int32))
    with pytest.raises(kdt.KdtError):
        kdt.kdt_radius_model_train(tree, cu(qs[:2048]), 8, epochs=1, gate=9)
    kdt.kdt_status(tree)
