"""Launch-shape autotuner for the batched engine.

Grid search on held-out samples of queries over the CTA width (1 to 32 warps per
query, i.e. 4 to 128 8-lane groups: threads / 8), CTAs per SM and tier-0 slab size, in
two stages (every shape on a small sample, the fastest few again on a batch of the
size the engine will run); every candidate must give the same results (they are
compared), the fastest is kept.
Results are persisted as JSON keyed by (graph fingerprint, GPU name, mode), so later
runs on the same graph and GPU reuse them without searching again (cache_path=None
searches every time and persists nothing).

The kernel is compiled for at most 32 registers per thread, so a CTA of T threads
fits min(2048 / T, 32) times per SM (32 resident CTAs at most); candidate CTA counts
are multiples of the SM count.  The frontier tile stays 8 diagonals: the expand
step's neighbour exchange is a shuffle inside an 8-lane group.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

from . import DeviceBatch, Engine, Graph, RESULT_DTYPE, default_config

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "gwfa_gb300", "autotune.json")


def fingerprint(graph: Graph, prune: bool) -> str:
    import torch
    info = graph.info()
    dev = torch.cuda.get_device_name(graph.device)
    return f"{dev}|V{info['n_vertices']}|E{info['n_arcs']}|B{info['total_bases']}|{'prune' if prune else 'exact'}"


def _time(engine: Engine, batch: DeviceBatch, max_lag: int, reps: int) -> float:
    import torch
    st = torch.cuda.current_stream()
    batch.run(engine, max_lag=max_lag)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        batch.run(engine, max_lag=max_lag)
        e1.record(st)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def _tier0_bytes(threads_ctas: int, log2: int, prune: bool) -> int:
    """Approximate device bytes of a tier of CTAs with 2^log2-tile slabs: per tile a
    hash line (64 / 128 bytes), a touched entry, three 16-byte list entries and one
    frontier snapshot (64 / 128 bytes); pruning adds the spill requests and T."""
    per_tile = (64 + 4 + 48 + 64) if not prune else (128 + 4 + 48 + 128 + 20 + 16)
    return threads_ctas * (per_tile << log2)


def _sweep(graph: Graph, batch: DeviceBatch, shapes, max_lag: int, reps: int, prune: bool):
    trials, ref = [], None
    fields = [f for f in RESULT_DTYPE.names if f != "device_us"]
    for th, per_sm, lg, ctas in shapes:
        cfg = default_config(graph, prune)
        cfg.threads = th
        cfg.tiers[0].threads = th
        cfg.tiers[0].ctas = ctas
        cfg.tiers[0].log2_tiles = lg
        eng = Engine(graph, prune=prune, config=cfg)
        ms = _time(eng, batch, max_lag, reps)
        res = batch.results()
        if ref is None:
            ref = res
        for f in fields:   # a launch shape must never change a result
            assert np.array_equal(res[f], ref[f]), (th, per_sm, lg, f)
        trials.append({"threads": th, "warps_per_query": th // 32, "ctas": ctas, "ctas_per_sm": per_sm,
                       "log2_tiles": lg, "ms": ms})
        eng.close()
    return trials


def autotune(graph: Graph, sample, max_lag: int = 0, threads=(32, 64, 128, 256, 384, 512, 768, 1024),
             per_sm_frac=(1.0,), log2_tiles=(15, 16), reps: int = 2,
             cache_path: str | None = DEFAULT_CACHE, force: bool = False, final_sample=None,
             keep: int = 5, max_tier0_bytes: int = 32 << 30) -> dict:
    """Best {threads, ctas, log2_tiles} for `graph` from a timing sweep.

    Stage 1 times every shape on `sample`; with `final_sample` (a held-out batch of
    the size the engine will run: a small sample is bound by its longest query, a
    full batch by throughput, and the best shape differs) the best shape of each CTA
    width within 4x of the fastest (at most `keep` widths) is timed again on it with
    `reps` repetitions and the best of those is chosen.
    Shapes whose tier-0 slabs would exceed max_tier0_bytes are skipped.  By default
    every shape fills the GPU (per_sm_frac 1.0): a persistent batch is bound by
    throughput, and a small sample cannot tell a half-filled GPU from a full one."""
    import torch
    prune = max_lag > 0
    key = fingerprint(graph, prune)
    if cache_path and not force and os.path.exists(cache_path):
        cache = json.load(open(cache_path))
        if key in cache:
            return cache[key]
    sms = torch.cuda.get_device_properties(graph.device).multi_processor_count
    shapes = []
    for th in threads:
        for frac in per_sm_frac:
            per_sm = max(1, int(min(2048 // th, 32) * frac))
            for lg in log2_tiles:
                lg = lg if not prune else lg - 1
                shape = (th, per_sm, lg, sms * per_sm)
                if shape not in shapes and _tier0_bytes(sms * per_sm, lg, prune) <= max_tier0_bytes:
                    shapes.append(shape)
    batch = DeviceBatch(sample, device=graph.device, order=np.argsort(-sample.lengths(), kind="stable").astype(np.uint32))
    trials = _sweep(graph, batch, shapes, max_lag, reps if final_sample is None else 1, prune)
    out = {"trials": trials, "sample_queries": len(sample), "when": time.time()}
    if final_sample is not None:
        # the best shape of each CTA width within 4x of the fastest: the small sample
        # is bound by its longest query and favours wide CTAs, a full batch by
        # throughput, so the final choice needs more than one width
        best_of = {}
        for t in sorted(trials, key=lambda t: t["ms"]):
            best_of.setdefault(t["threads"], t)
        fastest = min(t["ms"] for t in trials)
        top = [t for t in sorted(best_of.values(), key=lambda t: t["ms"]) if t["ms"] <= 4 * fastest][:keep]
        fb = DeviceBatch(final_sample, device=graph.device,
                         order=np.argsort(-final_sample.lengths(), kind="stable").astype(np.uint32))
        final = _sweep(graph, fb, [(t["threads"], t["ctas_per_sm"], t["log2_tiles"], t["ctas"]) for t in top],
                       max_lag, reps, prune)
        out["final_trials"] = final
        out["final_sample_queries"] = len(final_sample)
        out["best"] = min(final, key=lambda t: t["ms"])
    else:
        out["best"] = min(trials, key=lambda t: t["ms"])
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        cache = json.load(open(cache_path)) if os.path.exists(cache_path) else {}
        cache[key] = out
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return out


def apply(graph: Graph, tuned: dict, prune: bool = False):
    """Engine config with the tuned tier-0 launch shape."""
    b = tuned["best"]
    cfg = default_config(graph, prune)
    cfg.threads = b["threads"]
    cfg.tiers[0].threads = b["threads"]
    cfg.tiers[0].ctas = b["ctas"]
    cfg.tiers[0].log2_tiles = b["log2_tiles"]
    return cfg
