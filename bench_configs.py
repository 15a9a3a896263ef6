"""Secondary measurements of bench.py (--config ...): the other workloads,
each printed as one JSON line per measured form.  The contract line
(default config) is produced by bench.py itself."""
from __future__ import annotations

import json
import os
import math
import statistics
import time

import numpy as np


def _timer(torch):
    stream = torch.cuda.current_stream()

    def timeit(fn, reps=3, warm=1):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
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

    return timeit


def _exact(oracle, pts, qs, gi, gd, k, r=math.inf, n=64, seed=0):
    idx = np.sort(np.random.default_rng(seed).choice(len(qs), size=min(n, len(qs)), replace=False))
    wi, wd = oracle.knn_brute_threaded(pts, qs[idx], k, r)
    return bool(np.array_equal(gi[idx], wi) and np.array_equal(gd[idx].view(np.uint32), wd.view(np.uint32)))


def _emit(**kw):
    print(json.dumps(kw), flush=True)


def _peaks(kdt):
    """(measured HBM GB/s or the fallback, its source, L2 read GB/s from the library's probe)."""
    try:
        peaks = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")))
        hbm, src = float(peaks["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        hbm, src = 6800.0, "fallback"
    return hbm, src, kdt.kdt_l2_read_bandwidth(32 << 20, 200)


def _roofline(bytes_, ms, hbm, src, l2, note):
    ach = bytes_ / (ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "peak_source": src,
            "l2": {"peak": l2, "frac": ach / l2,
                   "peak_source": "L2 read bandwidth measured by the library's probe (32 MiB, L1-bypassing loads)"},
            "bytes": bytes_, "time": note}


def _loop(torch, fn, steps, warmup):
    """ms per call over `steps` calls after `warmup` untimed ones (CUDA events)."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(steps):
        fn()
    b.record(s)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def run_config(args):
    import torch

    import oracle
    from paper_2210_12859_gb300 import kdt, synth

    torch.cuda.set_device(0)
    timeit = _timer(torch)
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731

    if args.config == "uniform_small":
        pts, qs = synth.uniform_small()
        dp, dq = cu(pts), cu(qs)
        tree = kdt.kdt_build(dp)
        build_ms = timeit(lambda: kdt.kdt_rebuild(tree, dp, opts=kdt.KDT_BUILD_ASYNC), 5)
        for k in (1, 8):
            for name, fl in (("ordered", kdt.KDT_MORTON), ("unordered", kdt.KDT_MORTON | kdt.KDT_UNORDERED)):
                ms = timeit(lambda: kdt.kdt_knn(tree, dq, k, flags=fl), 5)
                gi, gd = kdt.kdt_knn(tree, dq, k, flags=fl)
                v = kdt.kdt_knn_visits(tree, dq, k, flags=fl).double().mean().item()
                wi, wd = oracle.knn_brute(pts, qs, k)
                _emit(config="uniform_small N=Q=2^14", form=f"{'fcp' if k == 1 else 'kNN k=8'} {name}",
                      query_qps=len(qs) / (ms / 1e3), query_ms=ms, build_ms=build_ms, visits_per_query=v,
                      bit_exact_full=bool(np.array_equal(gi.cpu().numpy().reshape(wi.shape), wi) and np.array_equal(
                          gd.cpu().numpy().reshape(wd.shape).view(np.uint32), wd.view(np.uint32))))
        return

    if args.config == "dims":
        n = 1 << 22
        sets = [(f"uniform D={D}", *synth.uniform_dim(n, n, D)) for D in (2, 4, 8)]
        sets.append(("surface D=3", *synth.surface_set(n, n)))
        for name, pts, qs in sets:
            dp, dq = cu(pts), cu(qs)
            tree = kdt.kdt_build(dp)
            build_ms = timeit(lambda: kdt.kdt_rebuild(tree, dp, opts=kdt.KDT_BUILD_ASYNC), 3)
            default_ms = timeit(lambda: kdt.kdt_knn(tree, dq, 16, flags=kdt.KDT_MORTON), 2)
            kdt.kdt_autotune(tree, dq, 16, kdt.KDT_MORTON)
            tuned = kdt.kdt_tuned_params(tree, 16)
            ms = timeit(lambda: kdt.kdt_knn(tree, dq, 16, flags=kdt.KDT_MORTON), 2)
            gi, gd = kdt.kdt_knn(tree, dq, 16, flags=kdt.KDT_MORTON)
            v = kdt.kdt_knn_visits(tree, dq, 16, flags=kdt.KDT_MORTON).double().mean().item()
            _emit(config="dims N=Q=2^22 kNN k=16 ordered", form=name, query_qps=n / (ms / 1e3), query_ms=ms,
                  default_launch_query_ms=default_ms,
                  launch_autotuned=dict(zip(("stage_levels", "claim_steps", "inline_depth", "light_run"), tuned)),
                  build_ms=build_ms, visits_per_query=v,
                  bit_exact_sample=_exact(oracle, pts, qs, gi.cpu().numpy(), gd.cpu().numpy(), 16))
            del tree
        return

    if args.config == "surface_learned":
        n = 1 << 24
        sh = synth.surface_shapes(256, synth.BASE_SEED + 4)
        pts = synth.surface_sample(sh, n, synth.BASE_SEED + 41)
        train = synth.surface_sample(sh, 1 << 20, synth.BASE_SEED + 42)
        qs = synth.surface_sample(sh, n, synth.BASE_SEED + 43)
        dp, dq, dt = cu(pts), cu(qs), cu(train)
        tree = kdt.kdt_build(dp)
        hbm, src, l2 = _peaks(kdt)
        F = kdt.KDT_MORTON
        gate_names = {kdt.KDT_GATE_ALL: "all", kdt.KDT_GATE_FAR: "far", kdt.KDT_GATE_NONE: "none"}
        for k, margin in ((8, 1.25), (32, 1.25), (8, 0.0), (32, 0.0)):
            # 1.25: the fixed margin of the configuration; 0: calibrated by the library
            kdt.kdt_autotune(tree, dq, k, F)
            t0 = time.perf_counter()
            loss = kdt.kdt_radius_model_train(tree, dt, k, epochs=40, seed=1, margin=margin, query_flags=F)
            train_s = time.perf_counter() - t0
            used_margin = kdt.kdt_radius_model_get(tree)[2]
            out_i = torch.empty((n, k), dtype=torch.int32, device="cuda")
            out_d = torch.empty((n, k), dtype=torch.float32, device="cuda")
            li = torch.empty_like(out_i)
            ld = torch.empty_like(out_d)
            steps, warm = max(args.steps, 5), max(args.warmup, 3)
            plain_ms = _loop(torch, lambda: kdt.kdt_knn(tree, dq, k, math.inf, F, out_i, out_d), steps, warm)
            learned_ms = _loop(torch, lambda: kdt.kdt_knn(tree, dq, k, math.inf, F | kdt.KDT_LEARNED, li, ld),
                               steps, warm)
            fb, ratio = kdt.kdt_learned_stats(tree)
            gated = kdt.kdt_learned_gated(tree)
            pv = kdt.kdt_knn_visits(tree, dq, k, flags=F).double().sum().item()
            lv = kdt.kdt_knn_visits(tree, dq, k, flags=F | kdt.KDT_LEARNED).double().sum().item()
            same = bool(torch.equal(li, out_i) and torch.equal(ld.view(torch.int32), out_d.view(torch.int32)))
            # forced gates, for context (the library keeps the fastest on the training queries)
            forced = {}
            kept = kdt.kdt_radius_model_gate(tree)
            for g in (kdt.KDT_GATE_ALL, kdt.KDT_GATE_FAR):
                if g == kept:
                    continue
                kdt.kdt_radius_model_set_gate(tree, g)
                forced[gate_names[g]] = plain_ms / _loop(
                    torch, lambda: kdt.kdt_knn(tree, dq, k, math.inf, F | kdt.KDT_LEARNED, li, ld), steps, warm)
            kdt.kdt_radius_model_set_gate(tree, kept)
            _emit(config="surface_learned N=Q=2^24 (256 spheres/tori)",
                  form=f"kNN k={k} plain vs learned ({'margin 1.25 as configured' if margin else 'calibrated margin'})",
                  margin=used_margin, gate=gate_names[kept], gated_queries=gated,
                  plain_qps=n / (plain_ms / 1e3), learned_qps=n / (learned_ms / 1e3),
                  speedup=plain_ms / learned_ms, speedup_with_other_gates=forced,
                  timing=f"{steps} calls of each form after {warm} warm-up calls",
                  fallback_rate=fb / n, radius_ratio=ratio,
                  plain_visits=pv / n, learned_visits=lv / n, identical=same, train_s=train_s, train_loss=loss,
                  roofline_plain=_roofline(n * (12 + 8 * k) + 16.0 * pv, plain_ms, hbm, src, l2, "plain query call"),
                  roofline_learned=_roofline(n * (12 + 8 * k) + 16.0 * lv + 16.0 * gated, learned_ms, hbm, src, l2,
                                             "learned query call (features and network included)"),
                  bit_exact_sample=_exact(oracle, pts, qs, out_i.cpu().numpy(), out_d.cpu().numpy(), k))
        return

    if args.config == "ablation":
        # the traversal choices around the stack-free machine, same results:
        # production kernel (inlined bottom subtrees, lane refill), the machine
        # as stated (one node per step), node after close subtree, stack-based
        forms = (("production", 0), ("stack-free, one node per step", kdt.KDT_PLAIN_STEP),
                 ("stack-free, node after close subtree", kdt.KDT_CLOSE_FIRST),
                 ("stack-based (explicit per-thread stack)", kdt.KDT_STACK))
        n = 1 << 24
        mix = synth.gmm_mixture(64, 3, 0.01, synth.BASE_SEED + 2)
        pts = synth.gmm_sample(mix, n, synth.BASE_SEED + 2)
        qs = synth.gmm_queries(mix, n, 0.1, synth.BASE_SEED + 3)
        rig_q = 10_000_000
        rig_pts = synth.uniform(1 << 22, 4, seed=synth.BASE_SEED + 6)
        rig_qs = synth.uniform(rig_q, 4, seed=synth.BASE_SEED + 7)
        cases = (("gmm_large N=Q=2^24 kNN k=8", pts, qs, 8, kdt.KDT_MORTON | kdt.KDT_COST_ORDER),
                 ("paper rig: uniform float4, N=2^22, Q=10^7, fcp", rig_pts, rig_qs, 1, kdt.KDT_MORTON),
                 ("paper rig: uniform float4, N=2^22, Q=10^7, kNN k=8", rig_pts, rig_qs, 8, kdt.KDT_MORTON))
        for cname, p_, q_, k, base in cases:
            dp, dq = cu(p_), cu(q_)
            tree = kdt.kdt_build(dp)
            ref_i, ref_d = kdt.kdt_knn(tree, dq, k, math.inf, base)
            out_i, out_d = torch.empty_like(ref_i), torch.empty_like(ref_d)
            kdt.kdt_autotune(tree, dq, k, base)
            tuned = kdt.kdt_tuned_params(tree, k)
            ms = timeit(lambda: kdt.kdt_knn(tree, dq, k, math.inf, base, out_i, out_d), 2)
            same = bool(torch.equal(out_i, ref_i) and torch.equal(out_d.view(torch.int32), ref_d.view(torch.int32)))
            _emit(config=cname, form="production, autotuned launch", query_qps=len(q_) / (ms / 1e3), query_ms=ms,
                  launch_autotuned=dict(zip(("stage_levels", "claim_steps", "inline_depth", "light_run"), tuned)),
                  identical_to_production=same)
            # the forms below run at the untuned defaults
            kdt.kdt_set_stage_levels(tree, 0)
            kdt.kdt_set_claim_steps(tree, 32 if k <= 1 else 64)
            kdt.kdt_set_inline_depth(tree, 2)
            kdt.kdt_set_light_run(tree, 1)
            for name, fl in forms:
                ms = timeit(lambda: kdt.kdt_knn(tree, dq, k, math.inf, base | fl, out_i, out_d), 2)
                same = bool(torch.equal(out_i, ref_i) and torch.equal(out_d.view(torch.int32), ref_d.view(torch.int32)))
                v = kdt.kdt_knn_visits(tree, dq, k, math.inf, base | fl).double().mean().item()
                _emit(config=cname, form=name, query_qps=len(q_) / (ms / 1e3), query_ms=ms, visits_per_query=v,
                      identical_to_production=same)
            del tree, dp, dq, ref_i, ref_d, out_i, out_d
        return

    if args.config == "range":
        # range queries (count -> offsets -> fill) and payload reductions on
        # the clustered distribution; hits compared with the oracle on samples
        n, nq = 1 << 24, 1 << 22
        mix = synth.gmm_mixture(64, 3, 0.01, synth.BASE_SEED + 2)
        pts = synth.gmm_sample(mix, n, synth.BASE_SEED + 2)
        qs = synth.gmm_queries(mix, nq, 0.1, synth.BASE_SEED + 8)
        dp, dq = cu(pts), cu(qs)
        tree = kdt.kdt_build(dp)
        r = 0.001
        F = kdt.KDT_MORTON
        sample = np.sort(np.random.default_rng(1).choice(nq, 48, replace=False))
        cnt_ms = timeit(lambda: kdt.kdt_radius_count(tree, dq, r, F), 3)
        counts = kdt.kdt_radius_count(tree, dq, r, F)
        off_ms = timeit(lambda: kdt.kdt_offsets(counts), 3)
        off, total = kdt.kdt_offsets(counts)
        fill_ms = timeit(lambda: kdt.kdt_radius_fill(tree, dq, r, off, total, True, F), 3)
        ids, d2 = kdt.kdt_radius_fill(tree, dq, r, off, total, True, F)
        kdt.kdt_status(tree)
        offh, idsh = off.cpu().numpy(), ids.cpu().numpy()
        _, woff, wids, _ = oracle.radius_brute(pts, qs[sample], r)
        ok = all(np.array_equal(np.sort(idsh[offh[q]:offh[q + 1]]), wids[woff[j]:woff[j + 1]])
                 for j, q in enumerate(sample))
        visits = kdt.kdt_radius_count(tree, dq, r, F | kdt.KDT_RANGE_VISITS).double().sum().item()
        # algorithmic bytes of the fill pass: query 12 B + 16 B per processed
        # node + 8 B per hit (id, d2) + 16 B of offsets, against measured HBM
        fill_bytes = nq * (12 + 16) + 16.0 * visits + 8.0 * total
        try:
            peaks = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")))
            hbm = float(peaks.get("hbm_gbs", 6800.0))
        except (OSError, ValueError):
            hbm = 6800.0  # the fallback peak when no measured peaks are available
        _emit(config=f"range: gmm N=2^24, Q=2^22 (90% mixture, 10% uniform), ball r={r}", form="ball count / offsets / fill",
              queries_per_s=nq / ((cnt_ms + off_ms + fill_ms) / 1e3), hits=int(total), hits_per_query=total / nq,
              hits_per_s=total / ((cnt_ms + off_ms + fill_ms) / 1e3), count_ms=cnt_ms, offsets_ms=off_ms,
              fill_ms=fill_ms, visits_per_query=visits / nq,
              roofline_fill={"bound": "hbm", "achieved": fill_bytes / (fill_ms / 1e3) / 1e9, "peak": hbm,
                             "unit": "GB/s", "frac": fill_bytes / (fill_ms / 1e3) / 1e9 / hbm,
                             "bytes_per_query": fill_bytes / nq},
              oracle_sample_sets_equal=ok)
        # long queries: r = 0.004 reaches ~1400 points and ~3900 nodes per query
        rl = 0.004
        lcnt_ms = timeit(lambda: kdt.kdt_radius_count(tree, dq, rl, F), 3)
        lcounts = kdt.kdt_radius_count(tree, dq, rl, F)
        loff, ltotal = kdt.kdt_offsets(lcounts)
        lfill_ms = timeit(lambda: kdt.kdt_radius_fill(tree, dq, rl, loff, ltotal, True, F), 3)
        lids, ld2 = kdt.kdt_radius_fill(tree, dq, rl, loff, ltotal, True, F)
        kdt.kdt_status(tree)
        lo_h = loff.cpu().numpy()
        lsample = sample[:16]
        _, lwoff, lwids, _ = oracle.radius_brute(pts, qs[lsample], rl)
        # only the sampled slices come back (the whole hit list is ~24 GB)
        lok = all(np.array_equal(np.sort(lids[int(lo_h[q]):int(lo_h[q + 1])].cpu().numpy()),
                                 lwids[lwoff[j]:lwoff[j + 1]]) for j, q in enumerate(lsample))
        del ld2
        lvisits = kdt.kdt_radius_count(tree, dq, rl, F | kdt.KDT_RANGE_VISITS).double().sum().item()
        lbytes = nq * (12 + 16) + 16.0 * lvisits + 8.0 * ltotal
        _emit(config=f"range: gmm N=2^24, Q=2^22 (90% mixture, 10% uniform), ball r={rl}",
              form="ball count / offsets / fill (long queries)", queries_per_s=nq / ((lcnt_ms + lfill_ms) / 1e3),
              hits=int(ltotal), hits_per_query=ltotal / nq, count_ms=lcnt_ms, fill_ms=lfill_ms,
              visits_per_query=lvisits / nq,
              roofline_count={"bound": "hbm", "achieved": (nq * 16 + 16.0 * lvisits) / (lcnt_ms / 1e3) / 1e9,
                              "peak": hbm, "unit": "GB/s",
                              "frac": (nq * 16 + 16.0 * lvisits) / (lcnt_ms / 1e3) / 1e9 / hbm},
              roofline_fill={"bound": "hbm", "achieved": lbytes / (lfill_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                             "frac": lbytes / (lfill_ms / 1e3) / 1e9 / hbm, "bytes_per_query": lbytes / nq},
              oracle_sample_sets_equal=lok)
        lo, hi = (dq - r).contiguous(), (dq + r).contiguous()
        bc_ms = timeit(lambda: kdt.kdt_box_count(tree, lo, hi, F), 3)
        bcounts = kdt.kdt_box_count(tree, lo, hi, F)
        boff, btotal = kdt.kdt_offsets(bcounts)
        bf_ms = timeit(lambda: kdt.kdt_box_fill(tree, lo, hi, boff, btotal, F), 3)
        bids = kdt.kdt_box_fill(tree, lo, hi, boff, btotal, F).cpu().numpy()
        bo = boff.cpu().numpy()
        _, wbo, wbi = oracle.box_brute(pts, qs[sample] - np.float32(r), qs[sample] + np.float32(r))
        okb = all(np.array_equal(np.sort(bids[bo[q]:bo[q + 1]]), wbi[wbo[j]:wbo[j + 1]]) for j, q in enumerate(sample))
        _emit(config=f"range: gmm N=2^24, Q=2^22, box half-width {r}", form="box count / offsets / fill",
              queries_per_s=nq / ((bc_ms + bf_ms) / 1e3), hits=int(btotal), hits_per_query=btotal / nq,
              count_ms=bc_ms, fill_ms=bf_ms, oracle_sample_sets_equal=okb)
        power = np.random.default_rng(2).random((n, 3)).astype(np.float32)  # photon power (RGB)
        kdt.kdt_tree_set_payload(tree, cu(power))
        red_ms = timeit(lambda: kdt.kdt_radius_reduce(tree, dq, r, kdt.KDT_REDUCE_DENSITY, F), 3)
        knn_ms = timeit(lambda: kdt.kdt_knn_reduce(tree, dq, 32, math.inf, kdt.KDT_REDUCE_DENSITY, F), 2)
        ko, kd = kdt.kdt_knn(tree, dq[torch.from_numpy(sample).cuda()], 32)
        want = oracle.knn_reduce(ko.cpu().numpy(), kd.cpu().numpy(), power, 2)
        got = kdt.kdt_knn_reduce(tree, dq, 32, math.inf, kdt.KDT_REDUCE_DENSITY, F).cpu().numpy()[sample]
        _emit(config="photon-map density (RGB power payload), gmm N=2^24, Q=2^22",
              form="fixed-radius gather (kdt_radius_reduce) / k=32 nearest (kdt_knn_reduce)",
              radius_reduce_qps=nq / (red_ms / 1e3), radius_reduce_ms=red_ms, knn_reduce_qps=nq / (knn_ms / 1e3),
              knn_reduce_ms=knn_ms, knn_reduce_equals_oracle_on_sample=bool(np.array_equal(got.view(np.uint32),
                                                                                            want.view(np.uint32))))
        return

    if args.config == "variants":
        # the other forms of the clustered 2^24 workload (fcp, k = 32 / 64, a
        # bounded radius) and the stored split dimension on surface data
        n = 1 << 24
        pts, qs = synth.gmm_large(n, n, seed=synth.BASE_SEED + 2)
        dp, dq = cu(pts), cu(qs)
        tree = kdt.kdt_build(dp)
        F = kdt.KDT_MORTON | kdt.KDT_COST_ORDER
        for k, r in ((1, math.inf), (32, math.inf), (64, math.inf), (8, 0.005)):
            kdt.kdt_autotune(tree, dq, k, F)
            gi, gd = kdt.kdt_knn(tree, dq, k, r, F)
            ms = timeit(lambda: kdt.kdt_knn(tree, dq, k, r, F, gi, gd), 2)
            v = kdt.kdt_knn_visits(tree, dq, k, r, F).double().mean().item()
            _emit(config="gmm_large N=Q=2^24", form=f"{'fcp' if k == 1 else f'kNN k={k}'}, r={r}",
                  query_qps=n / (ms / 1e3), query_ms=ms, visits_per_query=v,
                  launch_autotuned=dict(zip(("stage_levels", "claim_steps", "inline_depth", "light_run"),
                                            kdt.kdt_tuned_params(tree, k)),
                                        large_k_list=["shared heap", "global heap", "group of 4",
                                                      "group of 8"][kdt.kdt_large_k_list(tree, k)]),
                  bit_exact_sample=_exact(oracle, pts, qs, gi.cpu().numpy(), gd.cpu().numpy(), k, r, n=32))
            del gi, gd
        del tree, dp, dq
        sh = synth.surface_shapes(256, synth.BASE_SEED + 4)
        pts = synth.surface_sample(sh, n, synth.BASE_SEED + 41)
        qs = synth.surface_sample(sh, n, synth.BASE_SEED + 43)
        dp, dq = cu(pts), cu(qs)
        res = {}
        for name, opts in (("level split", 0), ("stored split dimension (widest extent)", kdt.KDT_BUILD_WIDEST)):
            tree = kdt.kdt_build(dp, opts=opts)
            gi, gd = kdt.kdt_knn(tree, dq, 8, math.inf, kdt.KDT_MORTON)
            ms = timeit(lambda: kdt.kdt_knn(tree, dq, 8, math.inf, kdt.KDT_MORTON, gi, gd), 3)
            v = kdt.kdt_knn_visits(tree, dq, 8, math.inf, kdt.KDT_MORTON).double().mean().item()
            res[name] = (gi.clone(), gd.clone())
            _emit(config="surface N=Q=2^24 kNN k=8", form=name, query_qps=n / (ms / 1e3), query_ms=ms,
                  visits_per_query=v,
                  identical_to_level_split=bool(torch.equal(gi, res["level split"][0]) and
                                                torch.equal(gd, res["level split"][1])))
            del tree
        return

    if args.config == "batched":
        c = synth.clouds(4096, seed=synth.BASE_SEED + 5)
        dp, dq = cu(c.points), cu(c.queries)
        Q = len(c.queries)
        t0 = time.perf_counter()
        forest = kdt.kdt_build_batched(dp, c.offsets)
        build_s = time.perf_counter() - t0
        out_i = torch.empty((Q, 8), dtype=torch.int32, device="cuda")
        out_d = torch.empty((Q, 8), dtype=torch.float32, device="cuda")
        res = {}
        # the library's batched-launch tuner (block size, claim steps), measured first
        th, cs, il, lr, _ = kdt.kdt_forest_autotune(forest, dq, c.qoffsets, 8, math.inf, kdt.KDT_MORTON, out_i, out_d)
        for name, fl in (("one persistent graph launch, Morton order", kdt.KDT_MORTON),
                         ("one persistent graph launch", 0),
                         ("one launch per tree", kdt.KDT_PER_TREE)):
            ms = timeit(lambda: kdt.kdt_knn_batched(forest, dq, c.qoffsets, 8, math.inf, fl, out_i, out_d), 2)
            res[name] = (ms, out_i.clone(), out_d.clone())
        same = all(torch.equal(res[a][1], res["one launch per tree"][1]) and
                   torch.equal(res[a][2], res["one launch per tree"][2]) for a in res)
        visits = kdt.kdt_knn_batched_visits(forest, dq, c.qoffsets, 8).double().sum().item()
        hbm, src, l2 = _peaks(kdt)
        # sampled oracle check on a few clouds
        gi = out_i.cpu().numpy()
        gd = out_d.cpu().numpy()
        ok = True
        for t in (0, 1000, 4095):
            p = c.points[c.offsets[t]:c.offsets[t + 1]]
            q = c.queries[c.qoffsets[t]:c.qoffsets[t + 1]]
            wi, wd = oracle.knn_brute(p, q[:64], 8)
            ok &= bool(np.array_equal(gi[c.qoffsets[t]:c.qoffsets[t] + len(wi)], wi))
        for name, (ms, _, _) in res.items():
            _emit(config=f"batched: 4096 clouds, {int(c.offsets[-1])} points, {Q} queries, kNN k=8", form=name,
                  query_qps=Q / (ms / 1e3), query_ms=ms, forest_build_s=build_s, identical_forms=same,
                  launch_autotuned={"threads": th, "claim_steps": cs, "inline_depth": il, "light_run": lr},
                  visits_per_query=visits / Q,
                  roofline=_roofline(Q * (12 + 8 * 8) + 16.0 * visits, ms, hbm, src, l2, "whole batched call"),
                  bit_exact_sample=ok)
        return
