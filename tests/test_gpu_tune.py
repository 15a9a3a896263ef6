"""Launch tuning never changes a result: every staging depth gives the same
bits; the autotuner picks one of its candidates and its choice survives a
save / load round trip."""
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


def test_autotune_and_tuning_file(kdt, tmp_path):
    pts, qs = synth.gmm_large(1 << 18, 1 << 16)
    tree = kdt.kdt_build(torch.from_numpy(pts).cuda())
    dq = torch.from_numpy(qs).cuda()
    lv, ms = kdt.kdt_autotune(tree, dq, 8, kdt.KDT_MORTON)
    assert lv in (0, 4, 6, 8, 10, 11, 12) and ms > 0
    path = os.path.join(tmp_path, "tuning.json")
    kdt.kdt_tuning_save(path)
    rows = json.load(open(path))
    assert any(r["D"] == 3 and r["log2n"] == 18 and r["stage_levels"] == lv for r in rows)
    kdt.kdt_tuning_load(path)
    a = kdt.kdt_knn(tree, dq, 8, flags=kdt.KDT_MORTON)
    kdt.kdt_set_stage_levels(tree, 0)
    b = kdt.kdt_knn(tree, dq, 8, flags=kdt.KDT_MORTON)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    open(path, "w").write('[\n  {"gpu": "x", "D": 3, "k_bucket": 3, "log2n": 18, "stage_levels": 99}\n]\n')
    with pytest.raises(kdt.KdtError):
        kdt.kdt_tuning_load(path)
