"""What the trained cost model gains over the plain scheduler, in batch time.

On a heavy-tailed batch (the large workload's query mix: lognormal 1-100 kb at
0.1-10% divergence, here on a 3 Mb graph of the same site mix) the plain schedule --
longest query first, every query starting on the small tier-0 slabs -- lets the heavy
queries overflow, and re-runs them on larger slabs at the end, where they form a
tail.  The learned plan predicts each query's hash memory and work from the six
features, routes the predicted overflows to large-slab CTAs that start at once, and
gives the few heaviest 1024-thread CTAs.  Both schedules must give identical results;
the learned one must be clearly faster and re-run fewer queries.
"""
import numpy as np
import pytest

import paper_2206_13574_gb300 as gw
from paper_2206_13574_gb300 import _build, costmodel, synth

pytestmark = pytest.mark.gpu


def _time(eng, batch, **kw):
    import torch
    batch.run(eng, **kw)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(2):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        batch.run(eng, **kw)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def test_learned_plan_beats_longest_first_in_time():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    c = synth.CONFIGS[4]
    g = synth.make_graph(synth.dataclasses.replace(c["graph"], backbone=3_000_000), 41)
    train = synth.make_queries(g, 1500, 41, c["length"], c["div"], c["weights"], c["loops"])
    test = synth.make_queries(g, 2000, 42, c["length"], c["div"], c["weights"], c["loops"])
    graph = gw.Graph.from_synth(g)
    model = gw.CostModel(graph, seed=1)
    feat, tgt, tres = costmodel.collect(model, gw.Engine(graph), train)
    coeffs = costmodel.time_coeffs(tres)
    costmodel.fit(model, feat, tgt, steps=1500, batch=256, lr=3e-3)

    # plain: longest first, all on tier 0, overflows re-run on the larger tiers
    plain_eng = gw.Engine(graph)
    bp = gw.DeviceBatch(test, order=np.argsort(-test.lengths(), kind="stable").astype(np.uint32))
    t_plain = _time(plain_eng, bp)
    r_plain = bp.results()
    retries_plain = int(plain_eng.last_retries()[0])
    plain_eng.close()

    # learned: predicted overflows on large-slab classes from the start
    cfg = gw.default_config(graph)
    cfg.wide.ctas, cfg.wide.log2_tiles, cfg.wide.threads = 1, 20, 512
    cfg.huge.ctas, cfg.huge.log2_tiles, cfg.huge.threads = 1, 23, 1024
    b0 = gw.DeviceBatch(test)
    pred = model.predict(model.features(b0)).cpu().numpy()
    order, n_huge, n_wide = gw.plan_schedule(pred, *costmodel.capacities(cfg))
    cfg.huge.ctas = max(1, min(n_huge, 32))
    cfg.wide.ctas = max(1, costmodel.wide_ctas(pred, order, n_wide, cfg.tiers[0].ctas, coeffs, first=n_huge))
    eng = gw.Engine(graph, config=cfg)
    bl = gw.DeviceBatch(test, order=order)
    t_learned = _time(eng, bl, n_wide=n_wide, n_huge=n_huge)
    r_learned = bl.results()
    retries_learned = int(eng.last_retries()[0])
    eng.close()

    for f in ("status", "edit_distance", "cells", "visited", "peak_frontier", "spills"):
        assert np.array_equal(r_plain[f], r_learned[f]), f
    assert retries_learned < retries_plain, (retries_learned, retries_plain)
    assert t_learned < 0.8 * t_plain, (t_learned, t_plain, n_huge, n_wide)
