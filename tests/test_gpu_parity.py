"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Distances and every work counter (n_scores, cells, peak frontier, visited,
spills, pruned, is_upper_bound) must be identical -- all of them are integers
fixed by Alg. 1-4, independent of execution order.  Exact distances are also
checked against the Eq. 1 DP.
"""
import ctypes
import json
import os

import numpy as np
import pytest

import oracle
import paper_2206_13574_gb300 as gw
from paper_2206_13574_gb300 import _build, synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "handtrace.json")
FIELDS = [("edit_distance", "distance"), ("n_scores", "n_scores"), ("cells", "cells"),
          ("peak_frontier", "peak"), ("visited", "visited"), ("spills", "spills"),
          ("pruned", "pruned"), ("is_upper_bound", "is_upper_bound")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    oracle.build()
    gw.load()


def _row(r) -> dict:
    if isinstance(r, dict):
        return r
    return {n: int(r[n]) for n in r.dtype.names}


def assert_same(r, w, ctx=""):
    r = _row(r)
    if w["distance"] < 0:
        assert r["status"] == w["distance"], (ctx, r, w)
        return
    assert r["status"] == 0, (ctx, r, w)
    for a, b in FIELDS:
        assert r[a] == w[b], (ctx, a, r[a], w[b], r, w)


def test_handtraced_cases_plain_and_batched():
    for c in json.load(open(GOLDEN))["cases"]:
        g = synth.Graph.from_lists(c["labels"], [tuple(a) for a in c["arcs"]])
        graph = gw.Graph.from_synth(g)
        q = c["q"].encode()
        ev = dict(evict_lag=c.get("evict_lag", 0), evict_every=c.get("evict_every", 0))
        r = graph.align(q, c["vs"], c["ve"], max_lag=c["a_diff"], **ev)
        exp = dict(c["expect"])
        exp.setdefault("pruned", 0)
        assert_same(r, exp, c["name"])
        assert r["evicted"] == exp.get("evicted", 0), c["name"]
        eng = gw.Engine(graph, prune=c["a_diff"] > 0)
        res = eng.align_batch(np.frombuffer(q, np.uint8), np.array([0, len(q)], np.uint64),
                              [c["vs"]], [c["ve"]], max_lag=c["a_diff"], **ev)
        assert_same(res[0], exp, c["name"] + "/batch")
        assert int(res[0]["evicted"]) == exp.get("evicted", 0), c["name"]


def test_config1_plain_one_launch_per_query():
    g, qs = synth.make_config(1)
    graph = gw.Graph.from_synth(g)
    want = oracle.gwfa_many(g, qs, range(len(qs)))
    dp = oracle.dp_many(g, qs, range(len(qs)))
    for i in range(len(qs)):
        r = graph.align(qs.query(i), int(qs.v_s[i]), int(qs.v_e[i]))
        assert_same(r, want[i], f"q{i}")
        assert r["edit_distance"] == dp[i]


def test_config1_batched():
    g, qs = synth.make_config(1)
    graph = gw.Graph.from_synth(g)
    eng = gw.Engine(graph)
    res = eng.align_batch(qs.seq, qs.off, qs.v_s, qs.v_e)
    want = oracle.gwfa_many(g, qs, range(len(qs)))
    for i in range(len(qs)):
        assert_same(res[i], want[i], f"q{i}")


def test_random_tiny_graphs_plain():
    for t in range(120):
        r = synth.Rng(2024, t)
        nv = r.one_int(1, 7)
        g = synth.random_small_graph(r, nv, 20, 0.3, t % 2 == 1)
        q = bytes(synth._ACGT[r.codes(r.one_int(0, 40))])
        vs = r.one_int(0, nv - 1)
        ve = r.one_int(vs, nv - 1)
        graph = gw.Graph.from_synth(g)
        w = oracle.gwfa(g, q, vs, ve)
        assert_same(graph.align(q, vs, ve), w, f"t{t}")
        graph.close()


def _sample(qs, k, seed):
    L = qs.lengths()
    order = np.argsort(L)
    pick = order[np.linspace(0, len(order) - 1, k).astype(np.int64)]
    return np.unique(pick)


def test_config2_full_batch_sampled():
    """The benchmark's workload (10k queries, default engine), oracle on a sample."""
    g, qs = synth.make_config(2)
    graph = gw.Graph.from_synth(g)
    eng = gw.Engine(graph)
    res = eng.align_batch(qs.seq, qs.off, qs.v_s, qs.v_e)
    assert np.all(res["status"] == 0)
    idx = _sample(qs, 240, 0)
    want = oracle.gwfa_many(g, qs, idx)
    for i, w in zip(idx, want):
        assert_same(res[i], w, f"q{i}")
    short = np.argsort(qs.lengths())[:30]
    dp = oracle.dp_many(g, qs, short)
    for i, d in zip(short, dp):
        assert int(res[i]["edit_distance"]) == d
    # every distance is bounded by the injected edits
    assert np.all(res["edit_distance"] <= qs.edits)


def test_batch_order_and_tiers_do_not_change_results():
    g, qs = synth.make_config(2, n_queries=300)
    graph = gw.Graph.from_synth(g)
    base = gw.Engine(graph).align_batch(qs.seq, qs.off, qs.v_s, qs.v_e)
    perm = np.random.default_rng(0).permutation(len(qs)).astype(np.uint32)
    # tiny first tier: most queries overflow and are re-run by the next tiers
    cfg = gw.default_config(graph)
    cfg.tiers[0].ctas = 64
    cfg.tiers[0].log2_tiles = 9
    cfg.tiers[1].ctas = 32
    cfg.tiers[1].log2_tiles = 13
    eng2 = gw.Engine(graph, config=cfg)
    res2 = eng2.align_batch(qs.seq, qs.off, qs.v_s, qs.v_e, order=perm)
    for f in gw.RESULT_DTYPE.names:
        if f != "device_us":   # wall time, not a result
            assert np.array_equal(base[f], res2[f]), f


@pytest.mark.parametrize("tiers", [3, 2, 1])
def test_concurrent_classes_do_not_change_results(tiers):
    """Huge and wide classes beside tier 0, all with small slabs so overflows cross
    from each class to the retry tiers; every counter equals the default engine's."""
    g, qs = synth.make_config(2, n_queries=300)
    graph = gw.Graph.from_synth(g)
    base = gw.Engine(graph).align_batch(qs.seq, qs.off, qs.v_s, qs.v_e)
    perm = np.random.default_rng(1).permutation(len(qs)).astype(np.uint32)
    cfg = gw.default_config(graph)
    cfg.n_tiers = tiers
    cfg.tiers[0].ctas, cfg.tiers[0].log2_tiles = 96, 10
    if tiers > 1:
        cfg.tiers[1].ctas, cfg.tiers[1].log2_tiles = 16, 13 if tiers > 2 else 18
    cfg.wide.ctas, cfg.wide.log2_tiles = 24, 11
    cfg.huge.ctas, cfg.huge.log2_tiles = 5, 12
    eng = gw.Engine(graph, config=cfg)
    res = eng.align_batch(qs.seq, qs.off, qs.v_s, qs.v_e, order=perm, n_huge=40, n_wide=60)
    assert eng.last_launches == tiers + 2 + 1   # tiers, both classes, the query packing
    if tiers == 1:   # no retry tier: overflows end as CAPACITY, the rest must match
        ok = res["status"] == 0
        assert np.all((res["status"] == 0) | (res["status"] == gw.GWFA_ERR_CAPACITY))
        assert ok.sum() > 100
    else:
        ok = np.ones(len(qs), dtype=bool)
        assert np.all(res["status"] == 0)
        assert eng.last_retries()[0] > 0
    for f in gw.RESULT_DTYPE.names:
        if f != "device_us":
            assert np.array_equal(base[f][ok], res[f][ok]), f


def test_1024_thread_ctas_do_not_change_results():
    """Tiers and the huge class at 1024 threads per CTA (half an SM each) give the same
    results as the default 512-thread engine."""
    g, qs = synth.make_config(2, n_queries=300)
    graph = gw.Graph.from_synth(g)
    base = gw.Engine(graph).align_batch(qs.seq, qs.off, qs.v_s, qs.v_e)
    cfg = gw.default_config(graph)
    cfg.tiers[0].ctas, cfg.tiers[0].threads = 96, 1024
    cfg.huge.ctas, cfg.huge.log2_tiles, cfg.huge.threads = 6, 18, 1024
    eng = gw.Engine(graph, config=cfg)
    order = np.argsort(-qs.lengths(), kind="stable").astype(np.uint32)
    res = eng.align_batch(qs.seq, qs.off, qs.v_s, qs.v_e, order=order, n_huge=12)
    for f in gw.RESULT_DTYPE.names:
        if f != "device_us":
            assert np.array_equal(base[f], res[f]), f


def test_capacity_error_without_retry_tier():
    g, qs = synth.make_config(2, n_queries=50)
    graph = gw.Graph.from_synth(g)
    cfg = gw.default_config(graph)
    cfg.n_tiers = 1
    cfg.tiers[0].ctas = 32
    cfg.tiers[0].log2_tiles = 8
    eng = gw.Engine(graph, config=cfg)
    res = eng.align_batch(qs.seq, qs.off, qs.v_s, qs.v_e)
    assert np.any(res["status"] == gw.GWFA_ERR_CAPACITY)
    ok = res["status"] == 0
    want = oracle.gwfa_many(g, qs, np.nonzero(ok)[0])
    for i, w in zip(np.nonzero(ok)[0], want):
        assert_same(res[i], w)


@pytest.mark.parametrize("a_diff", [30, 200])
def test_pruning_config2(a_diff):
    g, qs = synth.make_config(2, n_queries=160)
    graph = gw.Graph.from_synth(g)
    eng = gw.Engine(graph, prune=True)
    res = eng.align_batch(qs.seq, qs.off, qs.v_s, qs.v_e, max_lag=a_diff)
    want = oracle.gwfa_many(g, qs, range(len(qs)), a_diff=a_diff)
    for i, w in enumerate(want):
        assert_same(res[i], w, f"q{i}")
    assert np.any(res["is_upper_bound"] == 1)


def test_pruning_and_exact_cyclic_config3_small():
    g, _ = synth.make_config(3, n_queries=1, backbone=40000)
    c = synth.CONFIGS[3]
    qs = synth.make_queries(g, 24, 33, lambda r: 3000, c["div"], c["weights"], c["loops"])
    graph = gw.Graph.from_synth(g)
    ex = gw.Engine(graph).align_batch(qs.seq, qs.off, qs.v_s, qs.v_e)
    pr = gw.Engine(graph, prune=True).align_batch(qs.seq, qs.off, qs.v_s, qs.v_e, max_lag=100)
    wex = oracle.gwfa_many(g, qs, range(len(qs)))
    wpr = oracle.gwfa_many(g, qs, range(len(qs)), a_diff=100)
    for i in range(len(qs)):
        assert_same(ex[i], wex[i], f"exact q{i}")
        assert_same(pr[i], wpr[i], f"pruned q{i}")
        assert int(pr[i]["edit_distance"]) >= int(ex[i]["edit_distance"])


def test_edge_cases():
    g = synth.Graph.from_lists(["ACGTACGT", "GG", "T", "ACGTTTTTTTTTTTTTTTTTTTTTTTACG"],
                               [(0, 1), (1, 2), (0, 3), (3, 3)])
    graph = gw.Graph.from_synth(g)
    cases = [(b"", 0, 0), (b"", 0, 2), (b"ACGTACGTGGT", 0, 2), (b"ACGTACGT", 0, 0),
             (b"T", 2, 2), (b"ACGTACGTACGTTTTTTTTTTTTTTTTTTTTTTTTACGACGTTTTTTTT", 0, 3),
             (b"TTTT", 1, 0), (b"acgtacgtggt", 0, 2)]
    seq = b"".join(c[0] for c in cases)
    off = np.concatenate([[0], np.cumsum([len(c[0]) for c in cases])]).astype(np.uint64)
    eng = gw.Engine(graph)
    res = eng.align_batch(np.frombuffer(seq, np.uint8), off, [c[1] for c in cases],
                          [c[2] for c in cases])
    for i, (q, vs, ve) in enumerate(cases):
        w = oracle.gwfa(g, q, vs, ve)
        assert_same(res[i], w, f"case{i}")
        assert_same(graph.align(q, vs, ve), w, f"plain case{i}")
    # a base outside ACGT is rejected per query
    bad = eng.align_batch(np.frombuffer(b"ACGNT", np.uint8), np.array([0, 5], np.uint64), [0], [0])
    assert int(bad[0]["status"]) == gw.GWFA_ERR_INVALID
    # max_score stops the loop
    r = graph.align(b"TTTTTTTTTTTT", 0, 0, max_score=2)
    assert r["status"] == gw.GWFA_ERR_SCORE_LIMIT


def test_longest_queries_and_empty_batch():
    """100 kb queries (the longest of the lognormal workloads) against the oracle, on
    the batch and plain paths; an empty batch is a no-op."""
    c = synth.CONFIGS[4]
    g = synth.make_graph(synth.dataclasses.replace(c["graph"], backbone=400_000), 4)
    qs = synth.make_queries(g, 4, 41, synth._const(100_000), synth._const(0.004), c["weights"], c["loops"])
    graph = gw.Graph.from_synth(g)
    eng = gw.Engine(graph)
    res = eng.align_batch(qs.seq, qs.off, qs.v_s, qs.v_e)
    want = oracle.gwfa_many(g, qs, range(len(qs)))
    for i, w in enumerate(want):
        assert qs.lengths()[i] >= 100_000
        assert_same(res[i], w, f"long{i}")
    assert_same(graph.align(qs.query(0), int(qs.v_s[0]), int(qs.v_e[0])), want[0], "plain long0")
    empty = eng.align_batch(np.zeros(0, np.uint8), np.zeros(1, np.uint64), np.zeros(0, np.uint32),
                            np.zeros(0, np.uint32))
    assert len(empty) == 0


def test_device_batch_replays_as_cuda_graph():
    """The device-resident batch call (counter reset + tier launches, no host sync) is
    captured once into a CUDA graph and replayed; results match the direct call."""
    import torch
    g, qs = synth.make_config(2, n_queries=300)
    graph = gw.Graph.from_synth(g)
    eng = gw.Engine(graph)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        b = gw.DeviceBatch(qs, stream=st)
        b.run(eng, stream=st)          # sizes internal buffers outside the capture
    st.synchronize()
    direct = b.results()
    graph_obj = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph_obj, stream=st):
        b.run(eng, stream=torch.cuda.current_stream())
    for _ in range(2):
        b.out.zero_()
        graph_obj.replay()
        torch.cuda.synchronize()
        rep = b.results()
        for f in gw.RESULT_DTYPE.names:
            if f != "device_us":
                assert np.array_equal(rep[f], direct[f]), f


def test_autotuner_persists_and_keeps_results(tmp_path):
    from paper_2206_13574_gb300 import autotune
    g, qs = synth.make_config(2, n_queries=400)
    graph = gw.Graph.from_synth(g)
    sample = qs.subset(np.arange(0, 400, 2))
    path = str(tmp_path / "tune.json")
    t = autotune.autotune(graph, sample, threads=(256, 512), per_sm_frac=(1.0,), log2_tiles=(15, 16),
                          reps=1, cache_path=path)
    assert len(t["trials"]) == 4 and t["best"]["ms"] == min(x["ms"] for x in t["trials"])
    again = autotune.autotune(graph, sample, cache_path=path)      # served from the JSON cache
    assert again["best"] == t["best"]
    eng = gw.Engine(graph, config=autotune.apply(graph, t))
    rest = qs.subset(np.arange(1, 400, 2))
    res = eng.align_batch(rest.seq, rest.off, rest.v_s, rest.v_e)
    want = oracle.gwfa_many(g, rest, range(0, len(rest), 9))
    for i, w in zip(range(0, len(rest), 9), want):
        assert_same(res[i], w, f"q{i}")
