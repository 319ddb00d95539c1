"""Traceback (Alg. 5-6): the returned walk goes from v_s to v_e along arcs, its
spelled sequence is at exactly the reported distance from the query (several
optimal walks may exist, so validity is what is checked), and distance and work
counters equal those of the same run without traceback.  With lag pruning (Alg. 4)
the walk is the one the pruned wavefront reached the end along: the query aligns to
its spelled sequence with at most the reported (upper-bound) number of edits."""
import json
import os

import numpy as np
import pytest

import oracle
import paper_2206_13574_gb300 as gw
from paper_2206_13574_gb300 import _build, synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "handtrace.json")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    oracle.build()


def walk_distance(g, q: bytes, vs: int, ve: int, walk, arcs=None) -> int:
    """Levenshtein distance of the query to the walk's spelled sequence, after
    checking that the walk runs from vs to ve along arcs of g."""
    assert len(walk) >= 1 and walk[0] == vs and walk[-1] == ve
    arcs = arcs if arcs is not None else set(zip(g.arc_src.tolist(), g.arc_dst.tolist()))
    for a, b in zip(walk[:-1], walk[1:]):
        assert (int(a), int(b)) in arcs, (a, b)
    spelled = b"".join(g.label(int(v)) for v in walk)
    return oracle.levenshtein(spelled, q)


def check_walk(g, q: bytes, vs: int, ve: int, walk, d: int):
    assert walk_distance(g, q, vs, ve, walk) == d


def test_bubble_walk_is_the_unique_optimum():
    c = [x for x in json.load(open(GOLDEN))["cases"] if x["name"] == "bubble_spill_chain"][0]
    g = synth.Graph.from_lists(c["labels"], [tuple(a) for a in c["arcs"]])
    r, walk = gw.Graph.from_synth(g).align_path(c["q"].encode(), c["vs"], c["ve"])
    assert r["edit_distance"] == 0 and list(walk) == [0, 2, 3]


def test_plain_walks_config1_and_tiny_cyclic():
    g, qs = synth.make_config(1)
    graph = gw.Graph.from_synth(g)
    want = oracle.gwfa_many(g, qs, range(len(qs)))
    for i in range(len(qs)):
        r, walk = graph.align_path(qs.query(i), int(qs.v_s[i]), int(qs.v_e[i]))
        w = want[i]
        assert (r["edit_distance"], r["cells"], r["visited"], r["peak_frontier"]) == \
               (w["distance"], w["cells"], w["visited"], w["peak"])
        check_walk(g, qs.query(i), int(qs.v_s[i]), int(qs.v_e[i]), walk, r["edit_distance"])
    for t in range(60):
        rr = synth.Rng(77, t)
        nv = rr.one_int(2, 7)
        g2 = synth.random_small_graph(rr, nv, 12, 0.35, True)
        q = bytes(synth._ACGT[rr.codes(rr.one_int(1, 40))])
        gr = gw.Graph.from_synth(g2)
        r, walk = gr.align_path(q, 0, nv - 1)
        assert r["edit_distance"] == oracle.dp_distance(g2, q, 0, nv - 1)
        check_walk(g2, q, 0, nv - 1, walk, r["edit_distance"])
        gr.close()


def test_batched_walks_config2():
    import torch
    g, qs = synth.make_config(2, n_queries=200)
    graph = gw.Graph.from_synth(g)
    eng = gw.Engine(graph, prune=True)
    cap = 4096
    paths = torch.zeros(len(qs) * cap, dtype=torch.int32, device="cuda")
    plen = torch.zeros(len(qs), dtype=torch.int32, device="cuda")
    eng.set_paths(paths.data_ptr(), cap, plen.data_ptr())
    b = gw.DeviceBatch(qs)
    b.run(eng, traceback=True)
    torch.cuda.synchronize()
    res = b.results()
    exact = gw.Engine(graph).align_batch(qs.seq, qs.off, qs.v_s, qs.v_e)
    for f in ("status", "edit_distance", "cells", "visited", "peak_frontier", "spills"):
        assert np.array_equal(res[f], exact[f]), f
    P = paths.view(len(qs), cap).cpu().numpy()
    L = plen.cpu().numpy()
    for i in range(len(qs)):   # every walk
        assert 0 < L[i] <= cap
        check_walk(g, qs.query(i), int(qs.v_s[i]), int(qs.v_e[i]), P[i, :L[i]], int(res[i]["edit_distance"]))


def test_plain_walks_with_pruning_tiny_cyclic():
    """Traceback with pruning on the plain path: distance and counters equal the
    pruned oracle's, the walk is valid, and the query aligns to it within the
    reported upper bound (and not below the Eq. 1 distance)."""
    n_bounded = 0
    for t in range(80):
        rr = synth.Rng(78, t)
        nv = rr.one_int(2, 7)
        g2 = synth.random_small_graph(rr, nv, 12, 0.35, t % 2 == 1)
        q = bytes(synth._ACGT[rr.codes(rr.one_int(1, 40))])
        gr = gw.Graph.from_synth(g2)
        a_diff = rr.one_int(2, 12)
        r, walk = gr.align_path(q, 0, nv - 1, max_lag=a_diff)
        w = oracle.gwfa(g2, q, 0, nv - 1, a_diff=a_diff)
        assert (r["edit_distance"], r["cells"], r["visited"], r["pruned"], r["is_upper_bound"]) == \
               (w["distance"], w["cells"], w["visited"], w["pruned"], w["is_upper_bound"]), t
        lev = walk_distance(g2, q, 0, nv - 1, walk)
        assert oracle.dp_distance(g2, q, 0, nv - 1) <= lev <= r["edit_distance"], t
        n_bounded += r["is_upper_bound"]
        gr.close()
    assert n_bounded > 10   # pruning fired on many of them


def test_batched_walks_pruned_config3_full_graph():
    """Config 3 (the 1 Mb cyclic graph, 50 kb queries at 8% errors) lag-pruned at
    a_diff 1000 with traceback: the same distances and counters as without traceback
    (and as the oracle on a sample); every walk is valid and the query aligns to it
    within the reported upper bound -- in this workload exactly at it."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    g, qs = synth.make_config(3, n_queries=48)
    graph = gw.Graph.from_synth(g)
    eng = gw.Engine(graph, prune=True)
    cap = 8192
    paths = torch.zeros(len(qs) * cap, dtype=torch.int32, device="cuda")
    plen = torch.zeros(len(qs), dtype=torch.int32, device="cuda")
    eng.set_paths(paths.data_ptr(), cap, plen.data_ptr())
    b = gw.DeviceBatch(qs)
    b.run(eng, max_lag=1000, traceback=True)
    torch.cuda.synchronize()
    res = b.results()
    eng.set_paths(None)
    plain = eng.align_batch(qs.seq, qs.off, qs.v_s, qs.v_e, max_lag=1000)
    for f in ("status", "edit_distance", "cells", "visited", "peak_frontier", "spills", "pruned", "is_upper_bound"):
        assert np.array_equal(res[f], plain[f]), f
    for i, w in zip(range(0, len(qs), 8), oracle.gwfa_many(g, qs, range(0, len(qs), 8), a_diff=1000)):
        assert (int(res[i]["edit_distance"]), int(res[i]["cells"]), int(res[i]["pruned"])) == \
               (w["distance"], w["cells"], w["pruned"]), i
    assert res["is_upper_bound"].all()
    P = paths.view(len(qs), cap).cpu().numpy()
    L = plen.cpu().numpy()
    arcs = set(zip(g.arc_src.tolist(), g.arc_dst.tolist()))
    assert np.all((L > 0) & (L <= cap))
    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        lev = list(ex.map(lambda i: walk_distance(g, qs.query(i), int(qs.v_s[i]), int(qs.v_e[i]),
                                                  P[i, :L[i]], arcs), range(len(qs))))
    d = res["edit_distance"].astype(np.int64)
    assert np.all(np.array(lev) <= d)
    assert np.array_equal(np.array(lev), d)
