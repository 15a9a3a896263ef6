"""The benchmark's multi-rank timing helpers on CPU: two gloo ranks, barrier
and max over ranks (the path bench.py takes under torchrun, where each rank
is an independent replica with its own queries)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    w, r, lr = bench.dist_env()
    assert (w, r, lr) == (world, rank, rank)
    d = bench.dist_init(world, "gloo")
    bench.barrier(d)
    # each replica reports its own step time; the slowest rank defines the step
    m = bench.max_over_ranks(10.0 + rank, d)
    out.put((rank, m))
    bench.barrier(d)
    dist.destroy_process_group()


def test_two_rank_max_and_barrier():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 11.0), (1, 11.0)]


def test_single_rank_helpers_are_identity(monkeypatch):
    import bench

    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (1, 0, 0)
    assert bench.dist_init(1, "gloo") is None
    assert bench.max_over_ranks(3.5, None) == 3.5
    bench.barrier(None)


def test_four_rank_max_and_barrier():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 4, port, q)) for r in range(4)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(4))
    assert got == [(r, 13.0) for r in range(4)]


def test_replica_query_sets_are_distinct_and_reproducible():
    """Under torchrun each rank answers its own query set (weak scaling): the
    sets differ between ranks and are the same on every run."""
    import numpy as np

    from paper_2210_12859_gb300 import synth

    mix = synth.gmm_mixture(64, 3, 0.01, synth.BASE_SEED + 2)
    sets = [synth.gmm_queries(mix, 4096, 0.1, synth.BASE_SEED + 1000 + r) for r in (1, 2, 3)]
    again = synth.gmm_queries(mix, 4096, 0.1, synth.BASE_SEED + 1000 + 2)
    assert np.array_equal(sets[1], again)
    for a in range(3):
        for b in range(a + 1, 3):
            assert not np.array_equal(sets[a], sets[b])
