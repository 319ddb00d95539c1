"""Memory-bounded H~ (pruning mode) on the GPU: with eviction every counter --
distance, scores, cells, peak, insertions, pruned, spills and evictions -- equals the
oracle's; a lag beyond every a changes nothing; and a slab too small for a query's
unbounded H~ holds it once entries behind the lag are evicted."""
import numpy as np
import pytest

import oracle
import paper_2206_13574_gb300 as gw
from paper_2206_13574_gb300 import _build, synth

pytestmark = pytest.mark.gpu
FIELDS = [("edit_distance", "distance"), ("n_scores", "n_scores"), ("cells", "cells"),
          ("peak_frontier", "peak"), ("visited", "visited"), ("pruned", "pruned"), ("spills", "spills"),
          ("evicted", "evicted"), ("is_upper_bound", "is_upper_bound")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    oracle.build()


@pytest.fixture(scope="module")
def c3():
    g, qs = synth.make_config(3, n_queries=8, backbone=200_000)
    return g, qs, gw.Graph.from_synth(g)


def same(r, w, ctx):
    assert int(r["status"]) == 0, (ctx, r)
    for a, b in FIELDS:
        assert int(r[a]) == w[b], (ctx, a, int(r[a]), w[b])


@pytest.mark.parametrize("lag,every", [(300, 16), (1500, 64), (300, 1)])
def test_batched_parity_config3(c3, lag, every):
    g, qs, graph = c3
    eng = gw.Engine(graph, prune=True)
    res = eng.align_batch(qs.seq, qs.off, qs.v_s, qs.v_e, max_lag=300, evict_lag=lag, evict_every=every)
    want = oracle.gwfa_many(g, qs, range(len(qs)), a_diff=300, evict_lag=lag, evict_every=every)
    for i, w in enumerate(want):
        same(res[i], w, (lag, every, i))
    assert res["evicted"].sum() > 0


def test_plain_parity_and_huge_lag(c3):
    g, qs, graph = c3
    for i in range(3):
        args = (qs.query(i), int(qs.v_s[i]), int(qs.v_e[i]))
        r = graph.align(*args, max_lag=300, evict_lag=600, evict_every=32)
        same(r, oracle.gwfa(g, *args, a_diff=300, evict_lag=600, evict_every=32), i)
        free = graph.align(*args, max_lag=300)
        big = graph.align(*args, max_lag=300, evict_lag=10 ** 9, evict_every=8)
        for k in free:
            if k != "device_us":
                assert free[k] == big[k], (i, k)


def test_small_slab_fits_with_eviction(c3):
    import torch
    g, qs, graph = c3
    # tiles each query claims without the bound (engine statistics word 6)
    probe = gw.Engine(graph, prune=True)
    stats = torch.zeros(len(qs) * 8, dtype=torch.int64, device="cuda")
    probe.set_stats(stats.data_ptr())
    probe.align_batch(qs.seq, qs.off, qs.v_s, qs.v_e, max_lag=300)
    tiles = stats.view(len(qs), 8)[:, 6].cpu().numpy()
    probe.close()
    # a slab the largest query overflows: its load limit is 3/4 of the tiles
    log2 = int(np.ceil(np.log2(tiles.max() / 0.75))) - 1
    cfg = gw.default_config(graph, prune=True)
    cfg.n_tiers = 1
    cfg.tiers[0].ctas, cfg.tiers[0].log2_tiles = 8, log2
    eng = gw.Engine(graph, prune=True, config=cfg)
    free = eng.align_batch(qs.seq, qs.off, qs.v_s, qs.v_e, max_lag=300)
    bounded = eng.align_batch(qs.seq, qs.off, qs.v_s, qs.v_e, max_lag=300, evict_lag=300, evict_every=16)
    n_free = int((free["status"] == gw.GWFA_ERR_CAPACITY).sum())
    n_bounded = int((bounded["status"] == gw.GWFA_ERR_CAPACITY).sum())
    assert n_free > 0 and n_bounded < n_free, (log2, tiles.tolist(), n_free, n_bounded)


def test_config2_sample_parity():
    g, qs = synth.make_config(2, n_queries=120)
    graph = gw.Graph.from_synth(g)
    eng = gw.Engine(graph, prune=True)
    res = eng.align_batch(qs.seq, qs.off, qs.v_s, qs.v_e, max_lag=200, evict_lag=200, evict_every=8)
    idx = range(0, len(qs), 6)
    want = oracle.gwfa_many(g, qs, idx, a_diff=200, evict_lag=200, evict_every=8)
    for i, w in zip(idx, want):
        same(res[i], w, i)


def test_rejected_without_pruning_or_with_traceback(c3):
    g, qs, graph = c3
    with pytest.raises(gw.GwfaError):
        graph.align(qs.query(0), int(qs.v_s[0]), int(qs.v_e[0]), evict_lag=100)
    eng = gw.Engine(graph, prune=True)
    with pytest.raises(gw.GwfaError):
        eng.align_batch_device(1, 0, 0, 0, 0, None, None, 0, max_lag=100, evict_lag=100, traceback=True)
