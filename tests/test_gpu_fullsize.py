"""GPU parity at the stated sizes of the cyclic, large and serving workloads.

The CUDA path runs the full-size inputs (the 1 Mb cyclic graph with 50 kb queries at
8% insertion-biased errors; the 50 Mb graph with lognormal 1-100 kb queries at
0.1-10% divergence) and every distance and work counter of a seeded sample is
compared, element by element, with the oracle's Alg. 1-4 (Sec. 2.4-2.5; the exact
distances are Eq. 1's, to which exact Gwfa is pinned elsewhere):

* cyclic graph, lag-pruned with a_diff = 1000 (Alg. 4): 200 queries;
* cyclic graph, exact: 16 queries (each costs the oracle ~60 M cells), four of them
  also against Eq. 1's DP;
* cyclic graph, lag-pruned with the memory bound on H~ at the same lag: 100 queries;
* 50 Mb graph, exact: ~200 queries stratified over the whole divergence range and
  chosen within an oracle cell budget (estimated from the generator's injected edit
  counts, never from the GPU), run as one batch through the engine and, for the
  serving workload, as requests to the continuous-batching server.

Pruned results must also be upper bounds of the exact distance where both are known.
"""
import numpy as np
import pytest

import oracle
import paper_2206_13574_gb300 as gw
from paper_2206_13574_gb300 import _build, synth

pytestmark = pytest.mark.gpu
FIELDS = [("edit_distance", "distance"), ("n_scores", "n_scores"), ("cells", "cells"),
          ("peak_frontier", "peak"), ("visited", "visited"), ("spills", "spills"),
          ("pruned", "pruned"), ("is_upper_bound", "is_upper_bound"), ("evicted", "evicted")]


def same(r, w, ctx):
    assert int(r["status"]) == 0, (ctx, int(r["status"]))
    for a, b in FIELDS:
        assert int(r[a]) == w[b], (ctx, a, int(r[a]), w[b])


def seeded_sample(n_total: int, k: int, seed: int) -> np.ndarray:
    r = synth.Rng(seed, 99)
    return np.sort(np.argsort(r.u64(n_total), kind="stable")[:k])


def budget_sample(qs, per_bin: int, bins, max_cells: float, total_cells: float, seed: int) -> np.ndarray:
    """Queries spread over divergence bins, each under an oracle cost cap; the cost
    estimate (3 x injected edits^2 cells) comes from the generator alone."""
    est = 3.0 * qs.edits.astype(np.float64) ** 2
    r = synth.Rng(seed, 5)
    pri = r.u64(len(qs))
    pick = []
    for lo, hi in bins:
        idx = np.where((qs.divergence >= lo) & (qs.divergence < hi) & (est <= max_cells))[0]
        idx = idx[np.argsort(pri[idx], kind="stable")][:per_bin]
        pick.extend(idx.tolist())
    pick = np.array(sorted(pick), dtype=np.int64)
    keep = np.cumsum(est[pick]) <= total_cells
    return pick[keep]


@pytest.fixture(scope="module")
def c3():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    oracle.build()
    g, qs = synth.make_config(3)   # 1 Mb + loops, 2,000 x 50 kb, 8% errors (ins:del:sub 5:3:2)
    return g, qs, gw.Graph.from_synth(g), oracle.GraphArgs(g)


def test_config3_pruned_full_size(c3):
    g, qs, graph, ga = c3
    eng = gw.Engine(graph, prune=True)
    res = eng.align_batch(qs.seq, qs.off, qs.v_s, qs.v_e, max_lag=1000)
    assert np.all(res["status"] == 0)
    idx = seeded_sample(len(qs), 200, 3)
    want = oracle.gwfa_many(ga, qs, idx, a_diff=1000)
    for i, w in zip(idx, want):
        same(res[i], w, ("pruned", int(i)))
    eng.close()


def test_config3_exact_sample_and_upper_bound(c3):
    g, qs, graph, ga = c3
    idx = seeded_sample(len(qs), 16, 33)
    sub = qs.subset(idx)
    eng = gw.Engine(graph)
    res = eng.align_batch(sub.seq, sub.off, sub.v_s, sub.v_e)
    want = oracle.gwfa_many(ga, sub, range(len(sub)))
    for i, w in enumerate(want):
        same(res[i], w, ("exact", int(idx[i])))
    # and the definition itself (Eq. 1's DP over the co-reachable subgraph) on four
    dp = oracle.dp_many(ga, sub, range(4))
    assert [int(x) for x in res["edit_distance"][:4]] == dp
    eng.close()
    peng = gw.Engine(graph, prune=True)
    pr = peng.align_batch(sub.seq, sub.off, sub.v_s, sub.v_e, max_lag=1000)
    assert np.all(pr["edit_distance"] >= res["edit_distance"])   # pruning can only raise d
    peng.close()


def test_config3_pruned_with_memory_bound(c3):
    g, qs, graph, ga = c3
    idx = seeded_sample(len(qs), 100, 333)
    sub = qs.subset(idx)
    eng = gw.Engine(graph, prune=True)
    res = eng.align_batch(sub.seq, sub.off, sub.v_s, sub.v_e, max_lag=1000, evict_lag=1000, evict_every=64)
    want = oracle.gwfa_many(ga, sub, range(len(sub)), a_diff=1000, evict_lag=1000, evict_every=64)
    for i, w in enumerate(want):
        same(res[i], w, ("evict", int(idx[i])))
    assert res["evicted"].sum() > 0
    eng.close()


DIV_BINS = [(0.001, 0.01), (0.01, 0.03), (0.03, 0.06), (0.06, 0.101)]


@pytest.fixture(scope="module")
def c4():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    oracle.build()
    g, qs = synth.make_config(4, n_queries=4000)   # the 50 Mb graph, ~530k vertices
    idx = budget_sample(qs, 50, DIV_BINS, max_cells=2.5e7, total_cells=6e8, seed=4)
    sub = qs.subset(idx)
    want = oracle.gwfa_many(oracle.GraphArgs(g), sub, range(len(sub)))
    return g, sub, gw.Graph.from_synth(g), want


def test_config4_full_graph_sample(c4):
    g, sub, graph, want = c4
    assert len(sub) >= 180
    div = sub.divergence
    for lo, hi in DIV_BINS:   # every part of the 0.1-10% range is represented
        assert ((div >= lo) & (div < hi)).sum() >= 30, (lo, hi)
    assert sub.lengths().max() > 20_000 and div.max() > 0.09
    eng = gw.Engine(graph)
    res = eng.align_batch(sub.seq, sub.off, sub.v_s, sub.v_e,
                          order=np.argsort(-sub.lengths(), kind="stable"))
    for i, w in enumerate(want):
        same(res[i], w, ("c4", i))
    eng.close()


def test_config5_serving_on_the_full_graph(c4):
    g, sub, graph, want = c4
    srv = gw.Server(graph)
    tickets = []
    for i in range(len(sub)):
        while True:
            t = srv.submit(sub.query(i), int(sub.v_s[i]), int(sub.v_e[i]))
            if t is not None:
                break
        tickets.append(t)
    for i, t in enumerate(tickets):
        r = srv.wait(t, timeout_ms=120000)
        same(r, want[i], ("c5", i))
    srv.close()
