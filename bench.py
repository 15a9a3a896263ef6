"""Benchmark: kNN queries/s on one GB300 (or N replicas), one JSON line.

Workload (default): N = 2^24 3-D points from a 64-component isotropic Gaussian
mixture (sigma 0.01, centres uniform in [0,1]^3), Q = 2^24 queries (90% from
the mixture, 10% uniform in [0,1]^3); kNN with k = 8, unbounded radius,
ordered stack-free traversal with Morton query order.  One step = rebuild the
tree from the points + answer all Q queries (every stage of the single-tree
hot path).  The learned-radius form of the same query is timed beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank is an independent replica with its own query set
(queries shard across GPUs; the tree is rebuilt on every GPU), so per-GPU work
is fixed: weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "kNN queries/s, N=2^24 3-D k=8: plain vs learned-radius, bit-exact; % roofline"
K_NN = 8
LOG2N = 24


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--log2n", type=int, default=LOG2N, help="log2 of N = Q (default 24)")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the library's default launch parameters instead of running its tuner first "
                         "(profiling runs whose first traversal launch must be a full one)")
    ap.add_argument("--launch", default=None,
                    help="inline_depth,light_run,claim_steps set on the tree instead of running the tuner "
                         "(profiling runs that must capture the tuned kernel as the first traversal launch)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--config", default="gmm_large",
                    choices=["gmm_large", "uniform_small", "dims", "surface_learned", "batched", "ablation", "range",
                             "variants"],
                    help="gmm_large: the contract line; the others print one JSON line per measured form")
    return ap.parse_args()


# ---------------------------------------------------------------- distributed

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, backend):
    import torch.distributed as dist

    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist if world > 1 else None


def max_over_ranks(value: float, dist, device=None) -> float:
    """Max of a float over all ranks (identity without a process group)."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the
    timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[2 + i]
                          and "Not" not in r[2 + i]})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- CPU oracle

def cpu_oracle_qps(points, queries, k, n_queries, seed=5):
    """Oracle brute force (plain definition, all host cores) on a sample of the
    workload's queries against all N points; returns (queries/s, threads, sample)."""
    import oracle

    oracle.ensure_built()
    g = np.random.default_rng(seed)
    idx = np.sort(g.choice(len(queries), size=n_queries, replace=False))
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    ids, d2 = oracle.knn_brute_threaded(points, queries[idx], k, math.inf, threads)
    dt = time.perf_counter() - t0
    return n_queries / dt, threads, idx, ids, d2


def cpu_model() -> str:
    """The host CPU's model name (lscpu), else its architecture."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform

    return platform.machine()


def cpu_oracle_qps_1thread(points, queries, k, n_queries, seed=6):
    """The same brute force in one host thread, on a smaller sample of the
    workload's queries; returns queries/s."""
    import oracle

    oracle.ensure_built()
    g = np.random.default_rng(seed)
    idx = np.sort(g.choice(len(queries), size=n_queries, replace=False))
    t0 = time.perf_counter()
    oracle.knn_brute(points, queries[idx], k, math.inf)
    return n_queries / (time.perf_counter() - t0)


def reference_arm(args, world, rank):
    """The oracle timed as it stands on the host cores (rank 0 only)."""
    if rank != 0:
        return
    from paper_2210_12859_gb300 import synth

    n = 1 << args.log2n
    pts, qs = synth.gmm_large(n, n)
    per_step = 96 if args.log2n >= 24 else 512
    if args.warmup > 0:
        cpu_oracle_qps(pts, qs, K_NN, 16)
    times = []
    threads = os.cpu_count() or 1
    for s in range(args.steps):
        qps, threads, *_ = cpu_oracle_qps(pts, qs, K_NN, per_step, seed=100 + s)
        times.append(per_step / qps)
    ms = 1000.0 * statistics.median(times)
    value = per_step / (ms / 1000.0)
    sample = (f"{per_step} of the 2^{args.log2n} queries per step, brute force over all N points, threads over "
              "queries; value_1thread: 16 queries in one thread")
    one = cpu_oracle_qps_1thread(pts, qs, K_NN, 16)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args.log2n),
        "cpu_baseline": {"value": value, "unit": "queries/s", "cores": threads, "kind": "oracle", "sample": sample,
                         "value_1thread": one, "cpu": cpu_model()},
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(log2n):
    return {
        "workload": f"gmm_large: N=2^{log2n} 3-D float32 points, 64-component Gaussian mixture (sigma 0.01, "
                    f"centres U[0,1]^3); Q=2^{log2n} queries (90% mixture, 10% uniform [0,1]^3); kNN k=8, "
                    "max_radius=inf, ordered stack-free traversal, Morton query order with expensive queries first; "
                    "step = tree build + "
                    "all queries",
        "N": 1 << log2n, "Q": 1 << log2n, "D": 3, "k": K_NN,
        "cache": "inputs larger than L2 (tree 256 MiB, points and queries 192 MiB each, outputs 1 GiB)",
    }


# ---------------------------------------------------------------- profile data

KERNEL_SOURCES = ("kdt_traverse.cuh", "kdt_query_impl.cuh", "kdt_query.cuh")


def kernel_source_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2210_12859_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the traversal kernel from the committed ncu
    summary, or None when the kernel source changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "knn_kernel_gmm2p24_dram.txt")
    try:
        kv = dict(line.split(":", 1) for line in open(path) if ":" in line and not line.startswith("#"))
    except OSError:
        return None
    if kv.get("source_sha256_16", "").strip() != kernel_source_hash():
        return None
    try:
        return int(kv["traffic_bytes_per_launch"].strip())
    except (KeyError, ValueError):
        return None


# ---------------------------------------------------------------- our arm

def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, world, rank)
        return
    if args.config != "gmm_large":
        from bench_configs import run_config

        run_config(args)
        return

    import torch

    from paper_2210_12859_gb300 import kdt, synth

    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    dev = torch.device("cuda", local)
    n = 1 << args.log2n
    pts, qs = synth.gmm_large(n, n, seed=synth.BASE_SEED + 2)
    if rank > 0:  # each replica answers its own query set
        mix = synth.gmm_mixture(64, 3, 0.01, synth.BASE_SEED + 2)
        qs = synth.gmm_queries(mix, n, 0.1, synth.BASE_SEED + 1000 + rank)
    dp = torch.from_numpy(pts).to(dev)
    dq = torch.from_numpy(qs).to(dev)
    out_i = torch.empty((n, K_NN), dtype=torch.int32, device=dev)
    out_d = torch.empty((n, K_NN), dtype=torch.float32, device=dev)
    flags = kdt.KDT_MORTON | kdt.KDT_COST_ORDER
    tree = kdt.kdt_build(dp)
    stream = torch.cuda.current_stream()
    # the library's launch tuner (inline depth, claim steps, staging depth),
    # measured on 2^20 of the queries before anything is timed
    if args.launch:
        depth, light, claim = (int(x) for x in args.launch.split(","))
        kdt.kdt_set_inline_depth(tree, depth)
        kdt.kdt_set_light_run(tree, light)
        kdt.kdt_set_claim_steps(tree, claim)
    elif not args.no_tune:
        kdt.kdt_autotune(tree, dq, K_NN, flags)
    tuned = dict(zip(("stage_levels", "claim_steps", "inline_depth", "light_run"), kdt.kdt_tuned_params(tree, K_NN)))

    def step():
        kdt.kdt_rebuild(tree, dp, opts=kdt.KDT_BUILD_ASYNC)
        kdt.kdt_knn(tree, dq, K_NN, math.inf, flags, out_i, out_d)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    kdt.kdt_status(tree)

    # ---- timed region
    launches0 = kdt.kdt_launch_count()
    kdt.kdt_profile_enable(tree, True)
    barrier(dist)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(dist)
    ms_total = ev0.elapsed_time(ev1)
    trav_ms, trav_launches = kdt.kdt_profile_read(tree)
    kdt.kdt_profile_enable(tree, False)
    gpu_launches = kdt.kdt_launch_count() - launches0
    kdt.kdt_status(tree)
    ms_step = max_over_ranks(ms_total / args.steps, dist, dev)
    value = world * n / (ms_step / 1000.0)

    # ---- breakdown (untimed by the contract, reported for context)
    def timeit(fn, reps=2):
        ts = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    def timed_loop(fn):
        """ms per call over the contract's step count, after its warm-up."""
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / args.steps

    build_ms = timeit(lambda: kdt.kdt_rebuild(tree, dp, opts=kdt.KDT_BUILD_ASYNC), 3)
    query_ms = timeit(lambda: kdt.kdt_knn(tree, dq, K_NN, math.inf, flags, out_i, out_d), 2)
    visits = kdt.kdt_knn_visits(tree, dq, K_NN, math.inf, flags)
    v_sum = float(visits.double().sum().item())
    v_mean = v_sum / n

    # ---- sampled bit-exactness against the oracle (plain definition)
    res_i = out_i.cpu().numpy()
    res_d = out_d.cpu().numpy()
    exact = None
    cpu = None
    if rank == 0:
        qps_cpu, threads, idx, wi, wd = cpu_oracle_qps(pts, qs, K_NN, 256 if args.log2n >= 24 else 1024)
        exact = bool(np.array_equal(res_i[idx], wi) and np.array_equal(res_d[idx].view(np.uint32),
                                                                       wd.view(np.uint32)))
        cpu = {"value": qps_cpu, "unit": "queries/s", "cores": threads, "kind": "oracle",
               "sample": f"{len(idx)} random queries of the workload, brute force over all 2^{args.log2n} points "
                         "(plain definition, FP32), threads over queries; value_1thread: 16 queries in one thread",
               "value_1thread": cpu_oracle_qps_1thread(pts, qs, K_NN, 16), "cpu": cpu_model()}

    # ---- roofline of the dominant kernel (the traversal)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm = float(peaks["hbm_gbs"])
        peak_src = "measured"
    except Exception:
        hbm = 6800.0
        peak_src = "fallback"
    kern_ms = trav_ms / max(trav_launches, 1)
    bytes_per_launch = n * (4 * 3 + 8 * K_NN) + v_sum * 16.0
    achieved = bytes_per_launch / (kern_ms / 1000.0) / 1e9
    traffic = profiled_traffic()
    # the same algorithmic bytes against L2: the read bandwidth of a 32 MiB
    # buffer that stays in L2, measured by the library's own probe kernel
    l2_gbs = kdt.kdt_l2_read_bandwidth(32 << 20, 200)
    l2_note = "L2 read bandwidth measured by the library's probe (32 MiB buffer, 16-byte L1-bypassing loads)"
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "peak_source": peak_src,
                "kernel": "knn_kernel<layout0,K=8,ordered> (stack-free traversal)",
                "kernel_ms": kern_ms, "bytes_per_query": bytes_per_launch / n,
                "visits_per_query": v_mean,
                "l2": {"achieved": achieved, "peak": l2_gbs, "unit": "GB/s", "frac": achieved / l2_gbs,
                       "peak_source": l2_note}}

    # ---- learned radius form (same queries, same results)
    learned = None
    if not args.no_learned:
        mix = synth.gmm_mixture(64, 3, 0.01, synth.BASE_SEED + 2)
        train_q = torch.from_numpy(synth.gmm_queries(mix, 1 << 20, 0.1, synth.BASE_SEED + 77)).to(dev)
        t0 = time.perf_counter()
        # the gate (all queries, the far ones, none) is timed on the training
        # queries with the bench's query flags and the fastest kept
        loss = kdt.kdt_radius_model_train(tree, train_q, K_NN, epochs=40, seed=1, query_flags=flags)
        train_s = time.perf_counter() - t0
        gate = kdt.kdt_radius_model_gate(tree)
        li = torch.empty_like(out_i)
        ld = torch.empty_like(out_d)
        kdt.kdt_knn(tree, dq, K_NN, math.inf, flags | kdt.KDT_LEARNED, li, ld)
        # both query forms over the contract's step count, after its warm-up
        plain_loop_ms = timed_loop(lambda: kdt.kdt_knn(tree, dq, K_NN, math.inf, flags, out_i, out_d))
        learned_ms = timed_loop(lambda: kdt.kdt_knn(tree, dq, K_NN, math.inf, flags | kdt.KDT_LEARNED, li, ld))
        fb, ratio = kdt.kdt_learned_stats(tree)
        gated = kdt.kdt_learned_gated(tree)
        same = bool(torch.equal(li, out_i) and torch.equal(ld.view(torch.int32), out_d.view(torch.int32)))
        lv = kdt.kdt_knn_visits(tree, dq, K_NN, math.inf, flags | kdt.KDT_LEARNED)
        lv_sum = float(lv.double().sum().item())
        # algorithmic bytes: as the plain query, with the processed nodes of
        # the bounded and re-run passes, plus 16 B of features per gated query
        l_bytes = n * (4 * 3 + 8 * K_NN) + lv_sum * 16.0 + 16.0 * gated
        l_ach = l_bytes / (learned_ms / 1000.0) / 1e9
        learned = {"query_qps": n / (learned_ms / 1000.0), "query_ms": learned_ms,
                   "plain_query_qps": n / (plain_loop_ms / 1000.0), "plain_query_ms": plain_loop_ms,
                   "speedup_vs_plain": plain_loop_ms / learned_ms,
                   "timing": f"{args.steps} calls of each form after {args.warmup} warm-up calls, CUDA events",
                   "gate": {kdt.KDT_GATE_ALL: "all", kdt.KDT_GATE_FAR: "far", kdt.KDT_GATE_NONE: "none"}[gate],
                   "gated_queries": gated, "fallback_rate": fb / n, "radius_ratio": ratio,
                   "identical_to_plain": same, "visits_per_query": lv_sum / n, "train_s": train_s,
                   "train_loss": loss, "train_queries": 1 << 20, "train_epochs": 40,
                   "train_weighting": "plain-traversal work (resampled)",
                   "roofline": {"bound": "hbm", "achieved": l_ach, "peak": hbm, "unit": "GB/s", "frac": l_ach / hbm,
                                "bytes_per_query": l_bytes / n, "peak_source": peak_src,
                                "l2": {"peak": l2_gbs, "frac": l_ach / l2_gbs, "peak_source": l2_note},
                                "time": "whole learned call (Morton pass, features and network for the gated "
                                        "queries, bounded traversal)"}}

    # ---- the same queries on a tree with a stored per-node split dimension
    # (widest extent; the paper's other splitDimOf variant), same results
    widest = None
    if rank == 0:
        wtree = kdt.kdt_build(dp, opts=kdt.KDT_BUILD_WIDEST)
        wi = torch.empty_like(out_i)
        wd = torch.empty_like(out_d)
        w_build_ms = timeit(lambda: kdt.kdt_rebuild(wtree, dp, opts=kdt.KDT_BUILD_ASYNC), 2)
        w_ms = timeit(lambda: kdt.kdt_knn(wtree, dq, K_NN, math.inf, flags, wi, wd), 2)
        wv = kdt.kdt_knn_visits(wtree, dq, K_NN, math.inf, flags).double().mean().item()
        widest = {"query_qps": n / (w_ms / 1000.0), "query_ms": w_ms, "build_ms": w_build_ms,
                  "visits_per_query": wv, "speedup_vs_level_split": query_ms / w_ms,
                  "identical_to_plain": bool(torch.equal(wi, out_i) and torch.equal(wd.view(torch.int32),
                                                                                      out_d.view(torch.int32)))}
        kdt.kdt_status(wtree)
        wtree.free()

    # ---- end to end: host buffers in, host results out, through the C ABI
    e2e = None
    if not args.no_e2e:
        hp = torch.from_numpy(pts).pin_memory()
        hq = torch.from_numpy(qs).pin_memory()
        hi = torch.empty((n, K_NN), dtype=torch.int32).pin_memory()
        hd = torch.empty((n, K_NN), dtype=torch.float32).pin_memory()
        kdt.kdt_knn_host(hp, hq, K_NN, math.inf, flags, hi, hd)
        ts = []
        for _ in range(2):
            barrier(dist)
            t0 = time.perf_counter()
            kdt.kdt_knn_host(hp, hq, K_NN, math.inf, flags, hi, hd)
            ts.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(statistics.median(ts), dist, dev)
        e2e = {"value": world * n / e2e_s, "unit": "queries/s", "h2d_bytes_per_step": int(pts.nbytes + qs.nbytes),
               "d2h_bytes_per_step": int(hi.numel() * 4 + hd.numel() * 4), "seconds": e2e_s,
               "transfer": "pinned host buffers: points copied to the device, queries read and results written "
                           "in place by the query kernels through the host link",
               "identical": bool(np.array_equal(hi.numpy(), res_i))}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(args.log2n),
                           **{"launch_autotuned" if not (args.no_tune or args.launch) else "launch": tuned}),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
            "clocks": clk.summary(), "bit_exact_sample": exact,
            "breakdown": {"build_ms": build_ms, "query_ms": query_ms, "query_qps": n / (query_ms / 1000.0)},
            "learned": learned,
            "stored_split_dim": widest,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
