"""Open-loop load generation for the server: Poisson arrivals, p50/p99 latency.

run_server(): requests are submitted at their arrival times and completions are
polled in the same host loop (the server itself is the library's persistent
kernel); latency = completion time seen by the host - arrival time.

run_plain(): the baseline -- one synchronous single-query call (gwfa_align, one
kernel launch each) at a time, in arrival order; a request waits for every
earlier one.
"""
from __future__ import annotations

import time

import numpy as np


def _summary(lat: np.ndarray, bases: int, wall: float, n: int, done_at=None, arrivals=None) -> dict:
    out = {"requests": n, "p50_ms": float(np.percentile(lat, 50) * 1e3),
           "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
           "throughput_qps": n / wall, "gbp_per_s": bases / wall / 1e9, "wall_s": wall}
    if done_at is not None and n > 1:
        # the rate at which requests completed while they were still arriving: unlike
        # n / wall it is not set by the drain of the slowest requests after the last
        # arrival, so it tracks the offered rate until the server saturates
        window = float(arrivals[n - 1])
        out["sustained_qps"] = float((done_at <= window).sum()) / window if window > 0 else None
        out["window_s"] = window
    return out


def run_server(server, queries, arrivals: np.ndarray, idx=None) -> tuple[dict, list]:
    """Submit queries[idx[i]] at arrivals[i] (seconds from start); returns (summary, results)."""
    from . import RESULT_DTYPE
    idx = np.arange(len(arrivals)) if idx is None else np.asarray(idx)
    n = len(arrivals)
    qb = [queries.query(int(i)) for i in idx]
    vs = [int(queries.v_s[i]) for i in idx]
    ve = [int(queries.v_e[i]) for i in idx]
    tickets = np.zeros(n, dtype=np.uint64)
    out = np.zeros(n, dtype=RESULT_DTYPE)
    done = np.zeros(n, dtype=np.uint8)
    done_at = np.zeros(n)
    nxt = 0
    completed = 0
    t0 = time.perf_counter()
    while completed < n:
        now = time.perf_counter() - t0
        while nxt < n and arrivals[nxt] <= now:
            t = server.submit(qb[nxt], vs[nxt], ve[nxt])
            if t is None:            # ring full: retry on the next pass
                break
            tickets[nxt] = t
            nxt += 1
        if nxt:
            before = done[:nxt].copy()
            k = server.poll_many(tickets[:nxt], out[:nxt], done[:nxt])
            if k:
                t_done = time.perf_counter() - t0
                done_at[:nxt][(done[:nxt] == 1) & (before == 0)] = t_done
                completed += k
        if completed < n and nxt < n and nxt == completed:
            wait = arrivals[nxt] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(min(wait, 1e-3))
    wall = time.perf_counter() - t0
    lat = done_at - arrivals[:n]
    bases = int(sum(len(q) for q in qb))
    results = [{f: int(out[i][f]) for f in RESULT_DTYPE.names} for i in range(n)]
    return _summary(lat, bases, wall, n, done_at, arrivals), results


def run_plain(graph, queries, arrivals: np.ndarray, idx=None, max_lag: int = 0) -> tuple[dict, list]:
    """The same arrivals served by one synchronous gwfa_align call at a time."""
    idx = np.arange(len(arrivals)) if idx is None else np.asarray(idx)
    n = len(arrivals)
    done_at = np.zeros(n)
    results = []
    t0 = time.perf_counter()
    for k, i in enumerate(idx):
        now = time.perf_counter() - t0
        if arrivals[k] > now:
            time.sleep(arrivals[k] - now)
        results.append(graph.align(queries.query(int(i)), int(queries.v_s[i]), int(queries.v_e[i]),
                                   max_lag=max_lag))
        done_at[k] = time.perf_counter() - t0
    wall = time.perf_counter() - t0
    bases = int(sum(int(queries.lengths()[i]) for i in idx))
    return _summary(done_at - arrivals[:n], bases, wall, n), results
