"""Error paths reached without a device fault: injected allocation failures
(KDT_ENOMEM) and a lowered traversal step bound (KDT_ETRAVERSAL, reported by
kdt_status, visits -1); the library recovers and later calls are exact."""
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


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_injected_allocation_failures(kdt):
    pts, qs = synth.uniform_small(1 << 15, 4096)
    dp, dq = cu(pts), cu(qs)
    kdt.kdt_debug_fail_allocs(1)
    with pytest.raises(kdt.KdtError) as e:
        kdt.kdt_build(dp)
    assert e.value.code == kdt.KDT_ENOMEM
    tree = kdt.kdt_build(dp)
    ref = kdt.kdt_knn(tree, dq, 8, flags=kdt.KDT_MORTON)
    kdt.kdt_debug_fail_allocs(1)
    with pytest.raises(kdt.KdtError) as e:
        kdt.kdt_knn(tree, dq, 8, flags=kdt.KDT_MORTON)  # scratch for the Morton order
    assert e.value.code == kdt.KDT_ENOMEM
    got = kdt.kdt_knn(tree, dq, 8, flags=kdt.KDT_MORTON)
    assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])
    kdt.kdt_debug_fail_allocs(0)
    kdt.kdt_status(tree)


def test_step_bound_reports_traversal_error(kdt):
    pts, qs = synth.uniform_small(1 << 15, 4096)
    tree = kdt.kdt_build(cu(pts))
    dq = cu(qs)
    ref = kdt.kdt_knn(tree, dq, 8)
    ref_v = kdt.kdt_knn_visits(tree, dq, 8)
    # the bound is checked once per claim round: rounds of one step check it
    # after every step (a query descends about 15 levels, so all exceed 5)
    kdt.kdt_set_claim_steps(tree, 1)
    kdt.kdt_debug_set_step_cap(tree, 5)
    kdt.kdt_knn(tree, dq, 8)
    with pytest.raises(kdt.KdtError) as e:
        kdt.kdt_status(tree)
    assert e.value.code == kdt.KDT_ETRAVERSAL
    v = kdt.kdt_knn_visits(tree, dq, 8).cpu().numpy()
    assert np.all(v == -1)  # every query needs far more than 5 steps
    with pytest.raises(kdt.KdtError):
        kdt.kdt_status(tree)
    kdt.kdt_debug_set_step_cap(tree, 0)
    got = kdt.kdt_knn(tree, dq, 8)
    kdt.kdt_status(tree)
    assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])
    assert torch.equal(kdt.kdt_knn_visits(tree, dq, 8), ref_v)
    kdt.kdt_set_claim_steps(tree, -1)
