"""Serving: continuous batching over a resident graph.

Every result must be the same whether its request runs alone or arrives among
many others (tolerance 0: distance and every work counter), and equal to the
oracle's; a request that overflows a small hash slab is re-queued to a large one;
the kernel's bounded idle wait ends it and the next request starts it again.
"""
import time

import numpy as np
import pytest

import oracle
import paper_2206_13574_gb300 as gw
from paper_2206_13574_gb300 import _build, serving, synth

pytestmark = pytest.mark.gpu
KEYS = ("status", "edit_distance", "n_scores", "cells", "visited", "peak_frontier", "spills", "pruned",
        "is_upper_bound")


@pytest.fixture(scope="module")
def c2():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    g, qs = synth.make_config(2, n_queries=400)
    return g, qs, gw.Graph.from_synth(g)


def _same(a, b):
    return all(a[k] == b[k] for k in KEYS)


def test_alone_equals_in_the_mix_and_oracle(c2):
    g, qs, graph = c2
    cfg = gw.gwfa_server_config()
    gw.load().gwfa_server_default_config(graph.handle, cfg)
    cfg.ctas_small, cfg.ctas_big = 64, 8
    srv = gw.Server(graph, cfg)
    probe = [3, 17, 101, 250]
    alone = {}
    for i in probe:
        t = srv.submit(qs.query(i), int(qs.v_s[i]), int(qs.v_e[i]))
        alone[i] = srv.wait(t)
    # the same queries inside a stream of 300 others, submitted back to back
    tickets = {}
    order = list(range(300)) + probe + list(range(300, 400))
    for i in order:
        while True:
            t = srv.submit(qs.query(i), int(qs.v_s[i]), int(qs.v_e[i]))
            if t is not None:
                break
            time.sleep(1e-4)
        tickets.setdefault(i, []).append(t)
    mixed = {i: [srv.wait(t) for t in ts] for i, ts in tickets.items()}
    for i in probe:
        for r in mixed[i]:
            assert _same(r, alone[i]), (i, r, alone[i])
    want = oracle.gwfa_many(g, qs, probe + list(range(0, 400, 37)))
    for i, w in zip(probe + list(range(0, 400, 37)), want):
        r = mixed[i][0]
        assert r["status"] == 0 and r["edit_distance"] == w["distance"] and r["cells"] == w["cells"]
    st = srv.stats()
    assert st["completed"] == st["submitted"] == len(order) + len(probe)
    srv.close()


def test_overflow_requeues_to_large_slabs(c2):
    g, qs, graph = c2
    eng = gw.Engine(graph)
    ref = eng.align_batch(qs.seq, qs.off, qs.v_s, qs.v_e)
    cfg = gw.gwfa_server_config()
    gw.load().gwfa_server_default_config(graph.handle, cfg)
    cfg.ctas_small, cfg.log2_small = 32, 9          # too small for most queries
    cfg.ctas_big, cfg.log2_big = 16, 17
    cfg.big_length = 10 ** 9                        # admission sends everything to class 0
    srv = gw.Server(graph, cfg)
    ts = [srv.submit(qs.query(i), int(qs.v_s[i]), int(qs.v_e[i])) for i in range(120)]
    res = [srv.wait(t) for t in ts]
    for i, r in enumerate(res):
        assert r["status"] == 0
        for k in KEYS:
            assert r[k] == int(ref[i][k]), (i, k)
    assert srv.stats()["requeued"] > 0
    srv.close()


def test_model_admission_avoids_requeues(c2):
    """Admission by predicted memory: with a trained cost model attached, requests the
    model expects to overflow the small slabs go straight to the large ones, so fewer
    are re-queued than with length-only admission; results are unchanged."""
    from paper_2206_13574_gb300 import costmodel
    g, qs, graph = c2
    eng = gw.Engine(graph)
    model = gw.CostModel(graph, seed=3)
    feat, tgt, _ = costmodel.collect(model, eng, qs.subset(np.arange(200)))
    costmodel.fit(model, feat, tgt, steps=600, batch=128, lr=3e-3)
    test = list(range(200, 320))
    ref = eng.align_batch(qs.seq, qs.off, qs.v_s, qs.v_e)
    requeued = {}
    for name, m in (("length", None), ("model", model)):
        cfg = gw.gwfa_server_config()
        gw.load().gwfa_server_default_config(graph.handle, cfg)
        cfg.ctas_small, cfg.log2_small = 32, 11
        cfg.ctas_big, cfg.log2_big = 16, 17
        cfg.big_length = 10 ** 9                    # without a model: everything to class 0
        srv = gw.Server(graph, cfg, model=m)
        res = [srv.wait(srv.submit(qs.query(i), int(qs.v_s[i]), int(qs.v_e[i]))) for i in test]
        for i, r in zip(test, res):
            assert r["status"] == 0
            for k in KEYS:
                assert r[k] == int(ref[i][k]), (name, i, k)
        requeued[name] = srv.stats()["requeued"]
        srv.close()
    assert requeued["length"] > 0 and requeued["model"] < requeued["length"], requeued


def test_idle_exit_and_restart(c2):
    g, qs, graph = c2
    cfg = gw.gwfa_server_config()
    gw.load().gwfa_server_default_config(graph.handle, cfg)
    cfg.ctas_small, cfg.ctas_big = 16, 2
    cfg.idle_us = 2000                              # CTAs leave after ~2 ms without work
    srv = gw.Server(graph, cfg)
    a = srv.wait(srv.submit(qs.query(5), int(qs.v_s[5]), int(qs.v_e[5])))
    time.sleep(0.3)                                 # the kernel has ended by now
    b = srv.wait(srv.submit(qs.query(5), int(qs.v_s[5]), int(qs.v_e[5])))
    assert _same(a, b)
    assert srv.stats()["launches"] >= 2
    srv.close()


def test_poisson_stream_latency(c2):
    g, qs, graph = c2
    srv = gw.Server(graph)
    arr = synth.poisson_arrivals(2000.0, 0.15, seed=5)
    idx = np.arange(len(arr)) % len(qs)
    summ, res = serving.run_server(srv, qs, arr, idx)
    assert all(r["status"] == 0 for r in res)
    assert summ["p99_ms"] >= summ["p50_ms"] > 0
    srv.close()
