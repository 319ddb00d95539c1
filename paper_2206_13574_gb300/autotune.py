"""Launch-shape autotuner for the batched engine.

Grid search on a held-out sample of queries over the CTA width (2 to 16 warps per
query, i.e. 8 to 64 8-lane groups: threads / 8), CTAs per SM and tier-0 slab size; every candidate must
give the same results (they are compared), the fastest is kept.  Results are
persisted as JSON keyed by (graph fingerprint, GPU name, mode), so later runs on
the same graph and GPU reuse them without searching again.

The kernel is compiled for at most 32 registers per thread, so a CTA of T threads
fits 2048 / T times per SM; candidate CTA counts are multiples of the SM count.
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


def autotune(graph: Graph, sample, max_lag: int = 0, threads=(64, 128, 256, 512), per_sm_frac=(0.5, 1.0),
             log2_tiles=(15, 16), reps: int = 2, cache_path: str | None = DEFAULT_CACHE,
             force: bool = False) -> dict:
    """Best {threads, ctas, log2_tiles} for `graph` from a timing sweep on `sample`."""
    import torch
    prune = max_lag > 0
    key = fingerprint(graph, prune)
    if cache_path and not force and os.path.exists(cache_path):
        cache = json.load(open(cache_path))
        if key in cache:
            return cache[key]
    sms = torch.cuda.get_device_properties(graph.device).multi_processor_count
    order = np.argsort(-sample.lengths(), kind="stable").astype(np.uint32)
    batch = DeviceBatch(sample, device=graph.device, order=order)
    trials, ref = [], None
    for th in threads:
        for frac in per_sm_frac:
            per_sm = max(1, int(2048 // th * frac))
            for lg in log2_tiles:
                cfg = default_config(graph, prune)
                cfg.threads = th
                cfg.tiers[0].threads = th
                cfg.tiers[0].ctas = sms * per_sm
                cfg.tiers[0].log2_tiles = lg if not prune else lg - 1
                eng = Engine(graph, prune=prune, config=cfg)
                ms = _time(eng, batch, max_lag, reps)
                res = batch.results()
                fields = [f for f in RESULT_DTYPE.names if f != "device_us"]
                if ref is None:
                    ref = res
                for f in fields:   # a launch shape must never change a result
                    assert np.array_equal(res[f], ref[f]), (th, per_sm, lg, f)
                trials.append({"threads": th, "ctas": sms * per_sm, "log2_tiles": cfg.tiers[0].log2_tiles,
                               "ms": ms})
                eng.close()
    best = min(trials, key=lambda t: t["ms"])
    out = {"best": best, "trials": trials, "sample_queries": len(sample), "when": time.time()}
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
