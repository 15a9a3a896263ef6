"""The benchmark's command-line contract, on CPU.

The reference arm times the CPU oracle only, so it runs here in full at a
small size: one JSON line with the contract's keys, and nothing from ranks
other than 0.  The GPU arm must refuse to run without a GPU rather than fall
back to anything on the host.
"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(args, env_extra=None, timeout=600):
    env = dict(os.environ)
    for key in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(key, None)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=timeout)


def _json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def test_reference_arm_prints_one_contract_line():
    r = _bench(["--impl", "reference", "--steps", "2", "--warmup", "1", "--log2n", "12"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["steps"] == 2 and line["warmup"] == 1 and line["n_gpus"] == 1
    assert line["unit"] == "queries/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert "workload" in line["config"] and line["config"]["N"] == 1 << 12
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == line["value"] and cpu["sample"]
    assert cpu["value_1thread"] > 0 and cpu["cpu"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_cpu_oracle_helpers_time_the_oracle():
    """The GPU arm's CPU leg: the threaded brute force returns its sample and
    the oracle's results for it, and the one-thread figure is a rate."""
    import numpy as np

    import bench
    import oracle

    g = np.random.default_rng(1)
    pts = g.random((2000, 3)).astype(np.float32)
    qs = g.random((300, 3)).astype(np.float32)
    qps, threads, idx, wi, wd = bench.cpu_oracle_qps(pts, qs, 8, 40)
    assert qps > 0 and threads >= 1 and len(idx) == 40 and len(set(idx.tolist())) == 40
    bi, bd = oracle.knn_brute(pts, qs[idx], 8)
    assert np.array_equal(wi, bi) and np.array_equal(wd, bd)
    assert bench.cpu_oracle_qps_1thread(pts, qs, 8, 16) > 0


def test_reference_arm_other_ranks_exit_quietly():
    r = _bench(["--impl", "reference", "--steps", "1", "--warmup", "0", "--log2n", "10", "--gpus", "2"],
               {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert _json_lines(r.stdout) == []


def test_gpu_arm_refuses_to_run_without_a_gpu():
    import torch

    if torch.cuda.is_available():
        return
    r = _bench(["--steps", "1", "--warmup", "0", "--log2n", "10"])
    assert r.returncode != 0
    assert _json_lines(r.stdout) == []
    err = r.stderr.lower()
    assert "cuda" in err or "nvidia" in err, r.stderr[-2000:]
