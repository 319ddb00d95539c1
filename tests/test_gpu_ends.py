"""Formulation variants (Sec. 2.1: free walk start, free walk end, extension
without an end vertex) on the GPU, plain and batched: distances and every work
counter equal the oracle's variant Alg. 1-3, distances equal the variant Eq. 1 DP,
and a traceback walk is a walk of the graph whose own chain, aligned with the same
variant, costs the reported distance."""
import numpy as np
import pytest

import oracle
import paper_2206_13574_gb300 as gw
from oracle import EXTEND, FREE_END, FREE_START
from paper_2206_13574_gb300 import _build, synth

pytestmark = pytest.mark.gpu
VARIANTS = [FREE_START, FREE_END, FREE_START | FREE_END, EXTEND, EXTEND | FREE_START]
FIELDS = [("edit_distance", "distance"), ("n_scores", "n_scores"), ("cells", "cells"),
          ("peak_frontier", "peak"), ("visited", "visited"), ("spills", "spills")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    oracle.build()


def same(r, w, ctx):
    assert r["status"] == 0, (ctx, r, w)
    for a, b in FIELDS:
        assert int(r[a]) == w[b], (ctx, a, int(r[a]), w[b])


def trimmed(g, qs, seed):
    """The queries with a few bases cut from either end (fewer than the end
    vertices hold), so that free ends matter."""
    r = synth.Rng(seed, 0)
    seqs = []
    for i in range(len(qs)):
        q = qs.query(i)
        a = r.one_int(0, min(len(g.label(int(qs.v_s[i]))), len(q) // 4))
        b = r.one_int(0, min(len(g.label(int(qs.v_e[i]))), len(q) // 4))
        seqs.append(q[a:len(q) - b])
    off = np.zeros(len(seqs) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(x) for x in seqs])
    return synth.Queries(seq=np.frombuffer(b"".join(seqs), dtype=np.uint8).copy(), off=off,
                         v_s=qs.v_s.copy(), v_e=qs.v_e.copy(), edits=qs.edits.copy(),
                         divergence=qs.divergence.copy())


def check_walk(g, q, vs, ve, walk, d, ends):
    assert len(walk) >= 1 and walk[0] == vs
    if not ends & EXTEND:
        assert walk[-1] == ve
    arcs = set(zip(g.arc_src.tolist(), g.arc_dst.tolist()))
    for a, b in zip(walk[:-1], walk[1:]):
        assert (int(a), int(b)) in arcs
    chain = synth.Graph.from_lists([g.label(int(v)) for v in walk], [(i, i + 1) for i in range(len(walk) - 1)])
    chain_ends = (ends & FREE_START) | (FREE_END if ends & (FREE_END | EXTEND) else 0)
    assert oracle.dp_distance(chain, q, 0, len(walk) - 1, ends=chain_ends) == d


@pytest.mark.parametrize("ends", VARIANTS)
def test_plain_config1(ends):
    g, qs = synth.make_config(1)
    graph = gw.Graph.from_synth(g)
    tq = trimmed(g, qs, 5)
    for Q in (qs, tq):
        want = oracle.gwfa_many(g, Q, range(len(Q)), ends=ends)
        for i in range(len(Q)):
            r = graph.align(Q.query(i), int(Q.v_s[i]), int(Q.v_e[i]), ends=ends)
            same(r, want[i], (ends, i))
        for i in range(0, len(Q), 10):
            assert want[i]["distance"] == oracle.dp_distance(g, Q.query(i), int(Q.v_s[i]), int(Q.v_e[i]),
                                                             ends=ends)


@pytest.mark.parametrize("ends", VARIANTS)
def test_plain_tiny_graphs_and_walks(ends):
    for t in range(40):
        rr = synth.Rng(400 + ends, t)
        nv = rr.one_int(1, 7)
        g2 = synth.random_small_graph(rr, nv, 12, 0.35, t % 2 == 1)
        q = bytes(synth._ACGT[rr.codes(rr.one_int(0, 40))])
        vs = rr.one_int(0, nv - 1)
        ve = rr.one_int(vs, nv - 1)
        graph = gw.Graph.from_synth(g2)
        w = oracle.gwfa(g2, q, vs, ve, ends=ends)
        if w["distance"] < 0:
            graph.close()
            continue
        same(graph.align(q, vs, ve, ends=ends), w, (ends, t))
        r, walk = graph.align_path(q, vs, ve, ends=ends)
        assert r["edit_distance"] == w["distance"]
        check_walk(g2, q, vs, ve, walk, r["edit_distance"], ends)
        graph.close()


@pytest.mark.parametrize("ends", VARIANTS)
def test_batched_config2(ends):
    g, qs = synth.make_config(2, n_queries=300)
    Q = trimmed(g, qs, 9)
    graph = gw.Graph.from_synth(g)
    eng = gw.Engine(graph)
    res = eng.align_batch(Q.seq, Q.off, Q.v_s, Q.v_e, ends=ends)
    glob = eng.align_batch(Q.seq, Q.off, Q.v_s, Q.v_e)
    assert np.all(res["status"] == 0)
    assert np.all(res["edit_distance"] <= glob["edit_distance"])
    L = Q.lengths()
    idx = np.unique(np.argsort(L)[np.linspace(0, len(L) - 1, 40).astype(np.int64)])
    want = oracle.gwfa_many(g, Q, idx, ends=ends)
    for i, w in zip(idx, want):
        same(res[i], w, (ends, int(i)))


def test_batched_traceback_walks():
    import torch
    g, qs = synth.make_config(2, n_queries=200)
    Q = trimmed(g, qs, 11)
    graph = gw.Graph.from_synth(g)
    eng = gw.Engine(graph, prune=True)
    cap = 4096
    paths = torch.zeros(len(Q) * cap, dtype=torch.int32, device="cuda")
    plen = torch.zeros(len(Q), dtype=torch.int32, device="cuda")
    eng.set_paths(paths.data_ptr(), cap, plen.data_ptr())
    short = np.argsort(Q.lengths())[:15]
    for ends in (FREE_START | FREE_END, EXTEND | FREE_START):
        b = gw.DeviceBatch(Q)
        b.run(eng, traceback=True, ends=ends)
        torch.cuda.synchronize()
        res = b.results()
        exact = gw.Engine(graph).align_batch(Q.seq, Q.off, Q.v_s, Q.v_e, ends=ends)
        for f in ("status", "edit_distance", "cells", "visited", "peak_frontier", "spills"):
            assert np.array_equal(res[f], exact[f]), f
        P = paths.view(len(Q), cap).cpu().numpy()
        Ln = plen.cpu().numpy()
        for i in short:
            check_walk(g, Q.query(int(i)), int(Q.v_s[i]), int(Q.v_e[i]), P[i, :Ln[i]],
                       int(res[i]["edit_distance"]), ends)


def test_variants_rejected_where_unsupported():
    g, qs = synth.make_config(1, n_queries=4)
    graph = gw.Graph.from_synth(g)
    with pytest.raises(gw.GwfaError):
        graph.align(qs.query(0), int(qs.v_s[0]), int(qs.v_e[0]), max_lag=100, ends=FREE_END)
    with pytest.raises(gw.GwfaError):
        graph.align(qs.query(0), int(qs.v_s[0]), int(qs.v_e[0]), ends=8)
    eng = gw.Engine(graph, prune=True)
    with pytest.raises(gw.GwfaError):
        eng.align_batch(qs.seq, qs.off, qs.v_s, qs.v_e, max_lag=100, ends=FREE_START)
