"""Benchmark: aligned Gbp/s at bit-exact edit distance on the batched workload.

Workload (default): 1 Mb backbone graph, ~10.8k vertices, a site every ~200 bp
(SNP 70%, 1-50 bp indels 25%, 200-2000 bp alternate alleles 5%), 2-bit packed;
10,000 queries of log-uniform 1-20 kb length at U[0.5%, 5%] divergence, all in one
persistent launch (plus the overflow tiers), exact mode.

One step = the whole hot path over the batch: the alignment kernels with queries
packed and resident in HBM (`value`); `e2e` measures the same through the
host-buffer entry point (H2D of ASCII queries, packing kernel, alignment, D2H of
the results).  Queries are spread across ranks for N > 1 (weak scaling: every
rank aligns its own 10k-query batch; no collective on the data path).

`--impl reference` times the CPU oracle (Alg. 1-3 restated in C, one query per
thread on all host cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "aligned Gbp/s at bit-exact edit distance (batched)"
UNIT = "Gbp/s"
WORKLOAD = ("config2: 1 Mb backbone graph, 10k queries 1-20 kb log-uniform, 0.5-5% divergence, "
            "exact Gwfa, one persistent launch")


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def rank_queries(g, qs, rank: int):
    """Rank r's batch under weak scaling: rank 0 aligns the config-2 batch itself, rank
    r > 0 a batch of the same size and length / divergence distribution drawn with
    query seed 2 + 1000 r on the same graph, so every rank processes its own units."""
    if rank == 0:
        return qs
    from paper_2206_13574_gb300 import synth
    c = synth.CONFIGS[2]
    return synth.make_queries(g, len(qs), 2 + 1000 * rank, c["length"], c["div"], c["weights"], c["loops"])


def reduce_ranks(t_step: float, t_e2e: float, aligned_bp: int, cells: int, device) -> tuple:
    """Whole-job figures over the ranks: the slowest rank's step times (MAX) and the
    units all ranks processed (SUM).  One process: the inputs unchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t_step, t_e2e, aligned_bp, cells
    t = torch.tensor([t_step, t_e2e], dtype=torch.float64, device=device)
    u = torch.tensor([aligned_bp, cells], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(t[1]), int(u[0]), int(u[1])


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_reference(args, g, qs, sample_s: float, cores: int | None = None, keep: bool = False):
    """Time the oracle (Alg. 1-3 in C) on a bounded sample: one query per thread.
    With keep=True also return the sampled query ids and the oracle's results, so the
    run can check the GPU's results against them."""
    import oracle
    oracle.build()
    cores = cores or os.cpu_count() or 1
    rng = np.random.default_rng(12345)
    order = rng.permutation(len(qs))
    ga = oracle.GraphArgs(g)
    # grow the sample until it costs about `sample_s` seconds
    done, bases, t_total = 0, 0, 0.0
    chunk = max(cores * 8, 8)
    got = []
    t0 = time.perf_counter()
    while done < len(order) and time.perf_counter() - t0 < sample_s:
        idx = order[done:done + chunk]
        ts = time.perf_counter()
        res = oracle.gwfa_many(ga, qs, idx, threads=cores)
        t_total += time.perf_counter() - ts
        if keep:
            got.extend(res)
        bases += int(qs.lengths()[idx].sum())
        done += len(idx)
    out = {"value": bases / t_total / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{done} of {len(qs)} queries ({bases} bp), random order, "
                     f"{t_total:.1f} s wall on {cores} threads",
           "wall_s": t_total, "queries": done, "bases": bases}
    if keep:
        return out, order[:done], got
    return out


def cpu_dp_reference(g, qs, sample_s: float, cores: int | None = None) -> dict:
    """The dense Eq. 1 DP (the definition, over the co-reachable subgraph) timed on a
    bounded random sample on all host cores: the CPU cost of the problem without the
    wavefront method."""
    import oracle
    oracle.build()
    cores = cores or os.cpu_count() or 1
    order = np.random.default_rng(54321).permutation(len(qs))
    ga = oracle.GraphArgs(g)
    done, bases, t_total = 0, 0, 0.0
    t0 = time.perf_counter()
    while done < len(order) and time.perf_counter() - t0 < sample_s:
        idx = order[done:done + cores]
        ts = time.perf_counter()
        oracle.dp_many(ga, qs, idx, threads=cores)
        t_total += time.perf_counter() - ts
        bases += int(qs.lengths()[idx].sum())
        done += len(idx)
    return {"value": bases / t_total / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle (Eq. 1 DP)",
            "sample": f"{done} of {len(qs)} queries ({bases} bp), random order, {t_total:.1f} s wall on {cores} threads"}


VERIFY_FIELDS = (("edit_distance", "distance"), ("n_scores", "n_scores"), ("cells", "cells"),
                 ("peak_frontier", "peak"), ("visited", "visited"), ("spills", "spills"))


def verify(res, idx, want) -> dict:
    """GPU results against the oracle's on the sampled queries: distance and work counters."""
    bad = []
    for i, w in zip(idx, want):
        r = res[int(i)]
        if w["distance"] < 0:
            ok = int(r["status"]) == w["distance"]
        else:
            ok = int(r["status"]) == 0 and all(int(r[a]) == w[b] for a, b in VERIFY_FIELDS)
        if not ok:
            bad.append(int(i))
    return {"verified_queries": len(want), "mismatches": len(bad), "mismatch_ids": bad[:20],
            "fields": [a for a, _ in VERIFY_FIELDS]}


def tune_launch_shape(gw, graph, g, n_final: int) -> dict:
    """The autotuner's sweep of tier-0 launch shapes (warps per query, CTAs per SM,
    slab size) on held-out config-2 queries of the benchmark's length and divergence
    distribution drawn with other seeds: every shape on 1,000 queries, the best shape
    of each CTA width again on a batch of the benchmark's size; searched in every run."""
    from paper_2206_13574_gb300 import autotune, synth
    c = synth.CONFIGS[2]
    small = synth.make_queries(g, 1000, 22, c["length"], c["div"], c["weights"], c["loops"])
    full = synth.make_queries(g, n_final, 23, c["length"], c["div"], c["weights"], c["loops"])
    t0 = time.perf_counter()
    tuned = autotune.autotune(graph, small, log2_tiles=(15, 16, 17), reps=2, cache_path=None, final_sample=full)
    tuned["search_s"] = time.perf_counter() - t0
    tuned["sample"] = (f"stage 1: 1,000 held-out config-2 queries (seed 22); stage 2: the best shape of each CTA width within 4x of the fastest (at most 5) on "
                       f"{n_final:,} held-out queries (seed 23); longest first")
    return tuned


def learned_schedule(gw, graph, qs, ref, stream, flush, args, base_cfg=None) -> dict:
    """Cost model trained on logs of a separate config-2 batch (seed 12), then the
    benchmark batch run in the planned order with predicted overflows on large slabs."""
    import torch
    from paper_2206_13574_gb300 import costmodel, synth
    c2 = synth.CONFIGS[2]
    g_synth = synth.make_graph(c2["graph"], 2)          # the benchmark graph itself
    train_q = synth.make_queries(g_synth, 3000, 12, c2["length"], c2["div"], c2["weights"], c2["loops"])
    model = gw.CostModel(graph, seed=1)
    t0 = time.perf_counter()
    eng0 = gw.Engine(graph)
    feat, tgt, train_res = costmodel.collect(model, eng0, train_q)
    coeffs = costmodel.time_coeffs(train_res)
    eng0.close()
    costmodel.fit(model, feat, tgt, steps=1500, batch=512, lr=3e-3)
    t_train = time.perf_counter() - t0
    cfg = base_cfg if base_cfg is not None else gw.default_config(graph)
    # large-slab CTAs for the queries predicted to overflow tier 0; only as many are
    # launched as there are such queries, so tier 0 keeps the whole GPU otherwise
    cfg.wide.ctas, cfg.wide.log2_tiles, cfg.wide.threads = 152, 19, 512
    with torch.cuda.stream(stream):
        b = gw.DeviceBatch(qs, stream=stream)
        feat = model.features(b, stream=stream)
        pred = model.predict(feat, stream=stream)
    stream.synchronize()
    pred_np = pred.cpu().numpy()
    order, _, n_wide = gw.plan_schedule(pred_np, *costmodel.capacities(cfg))
    cfg.wide.ctas = max(1, costmodel.wide_ctas(pred_np, order, n_wide, cfg.tiers[0].ctas, coeffs))
    eng = gw.Engine(graph, config=cfg)
    with torch.cuda.stream(stream):
        b2 = gw.DeviceBatch(qs, order=order, stream=stream)
    ts = []
    for it in range(args.warmup + max(3, args.steps // 2)):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b2.run(eng, stream=stream, n_wide=n_wide)
        e1.record(stream)
        e1.synchronize()
        if it >= args.warmup:
            ts.append(e0.elapsed_time(e1) / 1e3)
    r = b2.results()
    assert np.array_equal(r["edit_distance"], ref["edit_distance"])
    retries = int(eng.last_retries()[0])
    t = float(np.mean(ts))
    ok = r["status"] == 0
    eng.close()
    return {"value": int(qs.lengths()[ok].sum()) / t / 1e9, "unit": UNIT, "ms_per_step": t * 1e3,
            "n_wide": n_wide, "tier0_overflows": retries, "train_s": t_train,
            "spearman_cells": costmodel.spearman(pred_np[:, 3], np.log1p(ref["cells"].astype(np.float64))),
            "train": "3000 other queries on the same graph (query seed 12), 1500 Adam steps on the GPU"}


def serving_run(gw, graph, qs, ref, rates=(2000.0, 20000.0), duration=0.5) -> dict:
    """p50/p99 latency and throughput of the continuous-batching server at two rates."""
    from paper_2206_13574_gb300 import serving, synth
    srv = gw.Server(graph)
    out = {}
    for lam in rates:
        arr = synth.poisson_arrivals(lam, duration, seed=int(lam))
        idx = np.arange(len(arr)) % len(qs)
        summ, res = serving.run_server(srv, qs, arr, idx)
        assert all(x["edit_distance"] == int(ref["edit_distance"][i]) for x, i in zip(res, idx))
        out[f"lambda_{int(lam)}"] = summ
    out["server"] = srv.stats()
    srv.close()
    return out


def ncu_case(args):
    """The benchmark kernel on a case small enough for a multi-pass ncu capture."""
    import torch
    import paper_2206_13574_gb300 as gw
    from paper_2206_13574_gb300 import _build, synth
    _build.build()
    g, qs = synth.make_config(2, n_queries=args.queries or 2000)
    graph = gw.Graph.from_synth(g)
    c = gw.default_config(graph)
    c.tiers[0].log2_tiles = 14
    c.tiers[1].ctas, c.tiers[1].log2_tiles = 16, 18
    c.tiers[2].ctas, c.tiers[2].log2_tiles = 1, 21
    eng = gw.Engine(graph, config=c)
    b = gw.DeviceBatch(qs, order=np.argsort(-qs.lengths(), kind="stable").astype(np.uint32))
    for _ in range(2):
        b.run(eng)
    torch.cuda.synchronize()
    r = b.results()
    retries = [int(x) for x in eng.last_retries()[:2]]
    eng.close()
    # after the captured launches: the same tier 0 alone, so that the work of the
    # captured tier-0 launch is known (queries that overflow it end as CAPACITY)
    c.n_tiers = 1
    e1 = gw.Engine(graph, config=c)
    b.run(e1)
    torch.cuda.synchronize()
    r1 = b.results()
    ok1 = r1["status"] == 0
    print(json.dumps({"ncu_case": True, "ok": int((r["status"] == 0).sum()),
                      "cells": int(r["cells"].sum()), "bases": int(qs.lengths().sum()), "retries": retries,
                      "tier0_completed": int(ok1.sum()), "tier0_completed_cells": int(r1["cells"][ok1].sum()),
                      # an overflowing query reports the cells it processed before it overflowed
                      "tier0_launch_cells": int(r1["cells"].sum()),
                      "tier0_overflows": int((r1["status"] == gw.GWFA_ERR_CAPACITY).sum())}))


def kernel_counters():
    """Per-cell counters of the alignment kernel from the committed ncu summary
    (profiles/align_kernel_counters.json), if they were taken on the current kernel
    source; else None: the counters no longer describe this kernel."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "align_kernel_counters.json")
    src = os.path.join(ROOT, "paper_2206_13574_gb300", "csrc", "gwfa_kernels.cu")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    return d if d.get("kernel_source_sha256") == sha else None


# Algorithmic bytes per cell (one live diagonal in one score) of the hot path, as the
# work-unit analysis counts them: GwfExtend reads the diagonal (12 B), one window of
# the query and of the label (8 B) and the vertex record (8 B) and writes the offset
# (4 B); GwfExpand makes up to 3 candidate merges and 2 probes of the old H~ (16 B
# each) and writes up to 3 frontier entries (12 B each) -- about 120 B -- plus 0.5 B
# per aligned base (2 bits of query and label each).
B_CELL = 120
# The kernel's own minimum (its design keeps the diagonal, the vertex record and the
# windows in registers and L1 and merges the frontier per 8-diagonal tile): the offset
# read and written by GwfExtend (8 B), the snapshot read and up to three candidates
# written by GwfExpand (16 B).
B_CELL_KERNEL = 24


def roofline(cells: int, aligned_bp: int, t_kernel: float, int_peak: dict | None, counters: dict | None,
             peak_gbs: float, peak_kind: str, steps: int) -> dict:
    alg = B_CELL * cells + 0.5 * aligned_bp
    achieved = alg / t_kernel / 1e9
    out = {"bound": "hbm", "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
           "frac": achieved / peak_gbs, "hbm_frac": achieved / peak_gbs,
           "traffic": None, "peak_kind": f"{peak_kind} HBM copy",
           "kernel": "align_kernel<exact> (all tiers of one step; CUDA events on its stream)",
           "bytes_per_cell": B_CELL, "bytes_per_aligned_base": 0.5,
           "kernel_bytes_per_cell": B_CELL_KERNEL,
           "hbm_frac_kernel_bytes": (B_CELL_KERNEL * cells + 0.5 * aligned_bp) / t_kernel / 1e9 / peak_gbs,
           "int_frac": None, "l2_frac": None}
    if counters:
        out["traffic"] = counters["dram_bytes_per_cell"] * cells
        out["traffic_note"] = ("ncu dram read+write per cell on the profiling case, scaled to this "
                               "step's cells: " + counters.get("source", ""))
        out["dram_bytes_per_cell_measured"] = counters["dram_bytes_per_cell"]
        out["l2_frac"] = counters["l2_throughput_pct"] / 100.0
        out["l2_note"] = "ncu lts__throughput (% of peak) of the profiled launch"
        out["warp_inst_per_cell"] = counters["warp_inst_per_cell"]
        out["alu_warp_inst_per_cell"] = counters["alu_warp_inst_per_cell"]
        if int_peak:
            rate = counters["alu_warp_inst_per_cell"] * cells / t_kernel
            out["int_achieved_warp_inst_per_s"] = rate
            out["int_peak_warp_inst_per_s"] = int_peak["warp_inst_per_s"]
            out["int_frac"] = rate / int_peak["warp_inst_per_s"]
            out["int_note"] = ("ALU-pipe warp instructions per cell (ncu) x cells / kernel time, against "
                               "the lop3 microbenchmark's ALU-pipe rate measured in this run")
    else:
        out["traffic_note"] = "no ncu counters for the current kernel source"
    if int_peak:
        out["int_peak"] = int_peak
    return out


def leg_config3() -> dict:
    """Cyclic graph with tandem-repeat loops, 2,000 x 50 kb at 8% errors: lag-pruned
    (a_diff 1000, all queries) against exact (200 queries), with the exact-match rate."""
    from paper_2206_13574_gb300 import experiments
    t0 = time.perf_counter()
    r = experiments.config3(n_pruned=2000, n_exact=200, a_diff=1000)
    r["leg_wall_s"] = time.perf_counter() - t0
    return r


def leg_config4(n: int) -> dict:
    """50 Mb graph, n lognormal 1-100 kb queries at 0.1-10% divergence, exact: the plain
    longest-first scheduler against the learned plan (cost model trained on config-2
    and config-3-graph logs)."""
    from paper_2206_13574_gb300 import experiments
    t0 = time.perf_counter()
    r = experiments.scheduler(n=n, n_plain=0, only=("plain_longest_first", "learned"))
    r["learned_vs_longest_first"] = r["plain_longest_first"]["s"] / r["learned"]["s"]
    r["leg_wall_s"] = time.perf_counter() - t0
    return r


def leg_config5(rates=(1000.0, 2000.0, 5000.0, 10000.0, 20000.0, 50000.0), max_requests: int = 20000,
                duration: float = 5.0) -> dict:
    """The 50 Mb graph resident in the continuous-batching server, Poisson arrivals at
    rising rates for `duration` seconds each (at most max_requests), until the server
    saturates: its sustained rate (requests completed while requests still arrive,
    per second) falls below 90% of the offered rate."""
    import paper_2206_13574_gb300 as gw
    from paper_2206_13574_gb300 import serving as sv
    from paper_2206_13574_gb300 import synth
    t0 = time.perf_counter()
    g, qs = synth.make_config(5, n_queries=4000)
    graph = gw.Graph.from_synth(g)
    cfg = gw.gwfa_server_config()
    gw.load().gwfa_server_default_config(graph.handle, cfg)
    cfg.log2_big = 22   # the heaviest config-5 queries hold ~10^7 diagonals
    srv = gw.Server(graph, cfg)
    out = {"workload": "config5: 50 Mb graph resident, lognormal 1-100 kb queries, 0.1-10% divergence, "
                       "Poisson arrivals", "server_config": {"ctas_small": cfg.ctas_small, "log2_small": cfg.log2_small,
                                                             "ctas_big": cfg.ctas_big, "log2_big": cfg.log2_big},
           "sweep": []}
    for lam in rates:
        arr = synth.poisson_arrivals(lam, min(duration, max_requests / lam), seed=int(lam))
        idx = np.arange(len(arr)) % len(qs)
        summ, _ = sv.run_server(srv, qs, arr, idx)
        summ["lambda"] = lam
        out["sweep"].append(summ)
        if summ["sustained_qps"] < 0.9 * lam:
            out["saturated_at_lambda"] = lam
            break
    out["max_sustained_qps"] = max(x["sustained_qps"] for x in out["sweep"])
    out["server"] = srv.stats()
    srv.close()
    graph.close()
    out["leg_wall_s"] = time.perf_counter() - t0
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gwfa", choices=["gwfa", "reference"])
    ap.add_argument("--queries", type=int, default=None, help="override the batch size")
    ap.add_argument("--cpu-sample-s", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-wide", type=int, default=0, help="queries on the wide CTA class")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the plain / learned / serving legs and the config 3-5 legs")
    ap.add_argument("--legs", default="3,4,5", help="config legs beside the headline (comma list, '' = none)")
    ap.add_argument("--c4-queries", type=int, default=5000)
    ap.add_argument("--plain-sample", type=int, default=300)
    ap.add_argument("--ncu-case", action="store_true",
                    help="small profiling case: --queries (default 2000) on ~3 GB of slabs, two batches")
    ap.add_argument("--int-peak-only", action="store_true", help="run the integer microbenchmark and exit")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    ws, rank, local = _dist()
    from paper_2206_13574_gb300 import synth
    if args.ncu_case:
        return ncu_case(args)
    if args.int_peak_only:
        import paper_2206_13574_gb300 as gw
        from paper_2206_13574_gb300 import _build
        _build.build()
        print(json.dumps(gw.measure_int_peak(local)))
        return
    g, qs = synth.make_config(2, n_queries=args.queries)
    total_bp = int(qs.lengths().sum())

    if args.impl == "reference":
        if rank != 0:
            return
        steps = []
        info = None
        for s in range(args.warmup + args.steps):
            r = cpu_reference(args, g, qs, sample_s=max(2.0, 30.0 / (args.warmup + args.steps)))
            if s >= args.warmup:
                steps.append(r)
                info = r
        # each step aligns a bounded random sample of the workload; the rate is the
        # sampled bases over the measured time of the timed steps
        wall = float(sum(r["wall_s"] for r in steps))
        v = float(sum(r["bases"] for r in steps)) / wall / 1e9
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": wall / len(steps) * 1e3,   # measured: one bounded sample per step
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
                "data": "synthetic", "config": {"workload": WORKLOAD, "queries": len(qs),
                                                "bases": total_bp,
                                                "per_step": (f"a random sample of {np.mean([r['queries'] for r in steps]):.0f} "
                                                             f"of the {len(qs)} queries "
                                                             f"({np.mean([r['bases'] for r in steps]):.0f} bp) per step; "
                                                             f"the whole batch at this rate would take "
                                                             f"{total_bp / (v * 1e9):.1f} s")},
                "cpu_baseline": dict(info, value=v),
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    import paper_2206_13574_gb300 as gw
    from paper_2206_13574_gb300 import _build
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _build.build()

    qs = rank_queries(g, qs, rank)
    total_bp = int(qs.lengths().sum())
    graph = gw.Graph.from_synth(g, device=local)
    from paper_2206_13574_gb300 import autotune
    tuned = tune_launch_shape(gw, graph, g, len(qs))
    tuned_cfg = autotune.apply(graph, tuned)
    eng = gw.Engine(graph, config=tuned_cfg)
    # longest queries first (a plain length-sorted schedule); the longest go to wide CTAs
    order = np.argsort(-qs.lengths(), kind="stable").astype(np.uint32)
    n_wide = max(args.n_wide, 0) if eng.config.wide.ctas else 0
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        batch = gw.DeviceBatch(qs, device=local, order=order, stream=stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # 256 MB > 129 MB L2
    torch.cuda.synchronize()

    def step():
        batch.run(eng, stream=stream, n_wide=n_wide)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    res = batch.results()
    launches_per_step = eng.last_launches
    int_peak = gw.measure_int_peak(local)   # integer ceiling of this GPU, this run

    clocks = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    times = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    t_step = float(np.mean(times))
    res_t = batch.results()
    assert np.array_equal(res_t["edit_distance"], res["edit_distance"])

    # end to end through the host-buffer entry point, inputs in pinned host memory
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_q = pin(qs.seq)
    h_off = pin(qs.off.view(np.int64))
    h_vs = pin(qs.v_s.view(np.int32))
    h_ve = pin(qs.v_e.view(np.int32))
    h_order = pin(order.view(np.int32))
    h_out = torch.empty(len(qs) * gw.RESULT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    lib = gw.load()
    opts = gw.gwfa_opts(0, 0, -1, 0, 0, 0, 0)
    import ctypes

    def e2e_step():
        st = lib.gwfa_align_batch(eng.handle, len(qs), h_q.data_ptr(), h_off.data_ptr(), h_vs.data_ptr(),
                                  h_ve.data_ptr(), h_order.data_ptr(), gw._sched(0, n_wide),
                                  ctypes.byref(opts),
                                  h_out.data_ptr(), stream.cuda_stream)
        assert st == 0, st

    for _ in range(2):
        e2e_step()
    e2e_times = []
    for _ in range(max(3, args.steps // 2)):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        stream.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        e2e_times.append(time.perf_counter() - t0)
    out_e2e = h_out.numpy().view(gw.RESULT_DTYPE)
    assert np.array_equal(out_e2e["edit_distance"], res["edit_distance"])
    t_e2e = float(np.mean(e2e_times))
    h2d = int(qs.seq.nbytes + qs.off.nbytes + qs.v_s.nbytes + qs.v_e.nbytes + order.nbytes)
    d2h = len(qs) * gw.RESULT_DTYPE.itemsize

    # bit-exactness checked in this run: the oracle's results on the CPU-baseline
    # sample against the GPU's, distance and work counters
    cpu, check = None, {"verified_queries": 0, "mismatches": 0,
                        "note": "no oracle sample in this run (--no-cpu-baseline or rank > 0)"}
    if rank == 0 and not args.no_cpu_baseline:
        cpu, vidx, vres = cpu_reference(args, g, qs, sample_s=args.cpu_sample_s, keep=True)
        check = verify(res, vidx, vres)
        one = cpu_reference(args, g, qs, sample_s=max(2.0, args.cpu_sample_s / 4), cores=1)
        cpu["single_core"] = {"value": one["value"], "unit": UNIT, "cores": 1, "sample": one["sample"]}
        cpu["dense_dp"] = cpu_dp_reference(g, qs, sample_s=max(2.0, args.cpu_sample_s / 3))
    ok = res["status"] == 0
    if check["mismatches"]:
        # an unverified batch: only the sampled queries that matched the oracle count
        good = np.zeros(len(qs), dtype=bool)
        good[np.setdiff1d(vidx, check["mismatch_ids"])] = True
        ok = ok & good
    aligned_bp = int(qs.lengths()[ok].sum())
    cells = int(res["cells"][ok].sum())
    # every rank's units and the slowest rank's times make the whole-job figures
    t_step, t_e2e, job_bp, job_cells = reduce_ranks(t_step, t_e2e, aligned_bp, cells, dev)
    value = job_bp / t_step / 1e9
    peak, peak_kind = _peaks()
    roof = roofline(cells, aligned_bp, t_step, int_peak, kernel_counters(), peak, peak_kind, args.steps)

    # S4: the plain path (one launch per query, synchronous) on a random sample
    plain = None
    if not args.no_extras:
        rng = np.random.default_rng(99)
        sidx = rng.choice(len(qs), size=min(args.plain_sample, len(qs)), replace=False)
        t0 = time.perf_counter()
        for i in sidx:
            r = graph.align(qs.query(int(i)), int(qs.v_s[i]), int(qs.v_e[i]))
            assert r["edit_distance"] == int(res["edit_distance"][i])
        tp = time.perf_counter() - t0
        pbp = int(qs.lengths()[sidx].sum())
        plain = {"value": pbp / tp / 1e9, "unit": UNIT, "sample": f"{len(sidx)} random queries",
                 "ms_per_query": tp / len(sidx) * 1e3}

    # S2: the learned schedule (cost model trained on a separate seeded batch)
    learned = None
    if not args.no_extras:
        learned = learned_schedule(gw, graph, qs, res, stream, flush, args, autotune.apply(graph, tuned))

    # S3: serving on the resident graph, Poisson arrivals
    serving_out = None
    if not args.no_extras:
        serving_out = serving_run(gw, graph, qs, res)

    eng.close()
    legs = {}
    if not args.no_extras and rank == 0:
        want = [x for x in args.legs.split(",") if x.strip()]
        if "3" in want:
            legs["config3"] = leg_config3()
        if "4" in want:
            legs["config4_scheduling"] = leg_config4(args.c4_queries)
        if "5" in want:
            legs["config5_serving"] = leg_config5()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "queries": len(qs), "bases": total_bp,
                       "aligned_bases": job_bp, "cells": job_cells,
                       "per_rank": "queries / bases are one rank's batch; aligned_bases and cells sum all ranks",
                       "parallelism": f"query-sharded x{ws} (replicated graph)",
                       "l2": "flushed (256 MB write) before every timed step",
                       "schedule": "longest query first", "n_wide": n_wide,
                       "wide": [eng.config.wide.ctas, eng.config.wide.log2_tiles, eng.config.wide.threads],
                       "engine_tiers": [
                           [eng.config.tiers[t].ctas, eng.config.tiers[t].log2_tiles,
                            eng.config.tiers[t].threads or eng.config.threads]
                           for t in range(eng.config.n_tiers)],
                       "threads_per_cta": eng.config.threads,
                       "launch_shape": dict(tuned["best"], source="autotuned (sweep below)"),
                       "autotune": {"trials": tuned["trials"], "final_trials": tuned.get("final_trials"),
                                    "sample": tuned["sample"], "search_s": tuned["search_s"]},
                       "ok_queries": int((res["status"] == 0).sum())},
            "verification": check,
            "e2e": {"value": job_bp / t_e2e / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": t_e2e * 1e3},
            "gpu_launches": launches_per_step * args.steps * ws,
            "roofline": roof,
            "cells_per_s": job_cells / t_step,
            # each edit removes at most one query base from the matched ones
            "matched_bases_per_s_lower_bound": float(np.maximum(
                qs.lengths()[ok] - res["edit_distance"][ok].astype(np.int64), 0).sum()) / t_step,
            "clocks": clk,
            "cpu_baseline": cpu,
            "plain": plain,
            "batched_vs_plain": (value / plain["value"]) if plain else None,
            "learned_schedule": learned,
            "serving": serving_out,
        }
        line.update(legs)
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
