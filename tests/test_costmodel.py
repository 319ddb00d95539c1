"""Learned cost model: CPU pins of the fp64 reference and the planner; GPU parity of
the feature, gradient and training kernels; the gain of the learned schedule."""
import os

import numpy as np
import pytest

import paper_2206_13574_gb300 as gw
from oracle import mlp_ref
from paper_2206_13574_gb300 import _build, synth

K = 16


def _codes(b: bytes) -> np.ndarray:
    lut = np.zeros(256, dtype=np.uint64)
    for ch, c in zip(b"ACGTacgt", [0, 1, 2, 3, 0, 1, 2, 3]):
        lut[ch] = c
    return lut[np.frombuffer(b, dtype=np.uint8)]


def _kmer(codes: np.ndarray, p: int) -> int:
    return int(sum(int(codes[p + t]) << (2 * t) for t in range(K)))


def coreachable_counts(g, vs: int, ve: int, n: int):
    """|S|, arcs inside S, vertices with >= 2 arcs inside S, arcs inside S on a cycle:
    S = vertices v with f(v) + |v| + b(v) <= ceil(1.25 n) + 64, f / b the shortest
    spelled lengths from v_s up to v / from after v to the end of v_e (Dijkstra)."""
    import heapq
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    budget = (5 * n + 3) // 4 + 64
    lens = g.lengths()
    arcs = np.unique(np.stack([g.arc_src.astype(np.int64), g.arc_dst.astype(np.int64)], 1), axis=0)
    out_adj, in_adj = {}, {}
    for u, w in arcs.tolist():
        out_adj.setdefault(u, []).append(w)
        in_adj.setdefault(w, []).append(u)

    def search(src, adj):
        dist = {src: 0}
        heap = [(0, src)]
        while heap:
            d, v = heapq.heappop(heap)
            if d > dist[v]:
                continue
            c = d + int(lens[v])
            if c > budget:
                continue
            for u in adj.get(v, []):
                if c < dist.get(u, budget + 1):
                    dist[u] = c
                    heapq.heappush(heap, (c, u))
        return dist

    f, b = search(vs, out_adj), search(ve, in_adj)
    S = {v for v in f if v in b and f[v] + int(lens[v]) + b[v] <= budget}
    nv = g.n_vertices
    m = csr_matrix((np.ones(len(arcs)), (arcs[:, 0], arcs[:, 1])), shape=(nv, nv))
    _, comp = connected_components(m, directed=True, connection="strong")
    inside = [(u, w) for u, w in arcs.tolist() if u in S and w in S]
    deg = np.bincount([u for u, _ in inside], minlength=nv) if inside else np.zeros(nv, np.int64)
    return len(S), len(inside), int((deg >= 2).sum()), sum(int(comp[u] == comp[w]) for u, w in inside)


def cpu_features(g, qs) -> np.ndarray:
    """The six raw features, computed the plain way."""
    kset = set()
    for v in range(g.n_vertices):
        c = _codes(g.label(v))
        for p in range(len(c) - K + 1):
            kset.add(_kmer(c, p))
    out = np.zeros((len(qs), 6), dtype=np.float64)
    for i in range(len(qs)):
        q = _codes(qs.query(i))
        n = len(q)
        miss = 0
        if n >= K:
            for t in range(64):
                miss += _kmer(q, t * (n - K) // 63) not in kset
        nverts, narcs, nbub, ncyc = coreachable_counts(g, int(qs.v_s[i]), int(qs.v_e[i]), n)
        out[i] = [np.log1p(n), miss / 64 if n >= K else 0.0, np.log1p(nverts), np.log1p(narcs),
                  nbub * 1000.0 / max(n, 1), np.log1p(ncyc)]
    return out


def shuffled_ids(g, qs, seed: int):
    """The same graph and queries with vertex ids permuted (ids no longer follow a
    topological order); every distance is unchanged."""
    r = np.random.default_rng(seed)
    perm = r.permutation(g.n_vertices)          # new id of old vertex v
    inv = np.argsort(perm)                      # old id of new vertex
    labels = [g.label(int(inv[v])) for v in range(g.n_vertices)]
    arcs = sorted(set(zip(perm[g.arc_src].tolist(), perm[g.arc_dst].tolist())))
    g2 = synth.Graph.from_lists(labels, arcs)
    q2 = synth.Queries(seq=qs.seq, off=qs.off, v_s=perm[qs.v_s].astype(np.uint32),
                       v_e=perm[qs.v_e].astype(np.uint32), edits=qs.edits, divergence=qs.divergence)
    return g2, q2


# ------------------------------------------------------------------ CPU pins


def test_reference_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    w = rng.normal(0, 0.3, mlp_ref.NPARAM)
    feat = rng.normal(0, 1, (40, 6))
    tgt = rng.normal(0, 1, (40, 4))
    args = (np.zeros(6), np.ones(6), np.zeros(4), np.ones(4))
    loss, g = mlp_ref.loss_and_grad(w, feat, tgt, *args, emulate_fp16=False)
    for i in rng.choice(mlp_ref.NPARAM, 60, replace=False):
        e = np.zeros_like(w)
        e[i] = 1e-6
        lp, _ = mlp_ref.loss_and_grad(w + e, feat, tgt, *args, emulate_fp16=False)
        lm, _ = mlp_ref.loss_and_grad(w - e, feat, tgt, *args, emulate_fp16=False)
        fd = (lp - lm) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_plan_schedule_orders_by_predicted_work_and_routes_big():
    _build.build()
    pred = np.zeros((6, 4), dtype=np.float32)
    pred[:, 3] = [3, 9, 1, 7, 5, 2]                 # log1p cells
    pred[:, 2] = [1, 1, 1, 20, 1, 21]                # log1p visited: queries 3 and 5 are huge
    order, n_huge, n_wide = gw.plan_schedule(pred, tier0_tiles=1000)
    assert (n_huge, n_wide) == (0, 2)
    assert list(order[:2]) == [3, 5]                 # big ones first, by predicted cells
    assert list(order[2:]) == [1, 4, 0, 2]           # the rest longest-predicted-first
    order, n_huge, n_wide = gw.plan_schedule(pred, tier0_tiles=10 ** 12)
    assert n_huge == 0 and n_wide == 0 and list(order) == [1, 3, 4, 0, 5, 2]
    # predicted tiles = expm1(visited) / 4: query 3 ~1.2e8, query 5 ~3.3e8; a 2e8 wide
    # class takes query 3 and leaves query 5 to the huge class, a 1e8 one takes neither
    order, n_huge, n_wide = gw.plan_schedule(pred, tier0_tiles=1000, wide_tiles=2 * 10 ** 8)
    assert (n_huge, n_wide) == (1, 1) and list(order[:2]) == [5, 3]
    order, n_huge, n_wide = gw.plan_schedule(pred, tier0_tiles=1000, wide_tiles=10 ** 8)
    assert (n_huge, n_wide) == (2, 0) and list(order[:2]) == [3, 5]


# ------------------------------------------------------------------ GPU


@pytest.fixture(scope="module")
def c2small():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    g, qs = synth.make_config(2, n_queries=600)
    graph = gw.Graph.from_synth(g)
    return g, qs, graph


@pytest.mark.gpu
def test_features_match_cpu(c2small):
    g, qs, graph = c2small
    sub = qs.subset(np.arange(0, 600, 10))
    m = gw.CostModel(graph)
    f = m.features(gw.DeviceBatch(sub)).cpu().numpy().astype(np.float64)
    ref = cpu_features(g, sub)
    assert np.array_equal(f[:, 1], ref[:, 1].astype(np.float32).astype(np.float64))   # k-mer misses exact
    assert np.allclose(f, ref, rtol=1e-5, atol=1e-5)


@pytest.mark.gpu
def test_features_on_shuffled_ids_follow_the_subgraph_not_the_ids():
    """With vertex ids permuted, the id interval [v_s, v_e] no longer describes the
    s -> e subgraph; the co-reachable counts do not depend on the ids at all."""
    g0, q0 = synth.make_config(3, n_queries=40, backbone=120_000)   # cyclic: loops count
    g, qs = shuffled_ids(g0, q0, seed=5)
    m = gw.CostModel(gw.Graph.from_synth(g))
    f = m.features(gw.DeviceBatch(qs)).cpu().numpy().astype(np.float64)
    ref = cpu_features(g, qs)
    assert np.allclose(f, ref, rtol=1e-5, atol=1e-5)
    m0 = gw.CostModel(gw.Graph.from_synth(g0))
    f0 = m0.features(gw.DeviceBatch(q0)).cpu().numpy().astype(np.float64)
    assert np.array_equal(f0, f)                    # the same subgraphs under either numbering
    span = np.abs(qs.v_e.astype(np.int64) - qs.v_s.astype(np.int64)) + 1
    assert (np.log1p(span) != ref[:, 2]).mean() > 0.9   # what the id interval would have counted
    assert ref[:, 5].max() > 0                          # loop arcs found


@pytest.mark.gpu
def test_gradient_matches_fp64_reference(c2small):
    import torch
    g, qs, graph = c2small
    m = gw.CostModel(graph, seed=3)
    eng = gw.Engine(graph)
    from paper_2206_13574_gb300 import costmodel
    feat, tgt, _ = costmodel.collect(m, eng, qs.subset(np.arange(200)))
    f = feat.double()
    t = tgt.double()
    norm = [f.mean(0).cpu().numpy(), f.std(0).clamp_min(1e-3).cpu().numpy(),
            t.mean(0).cpu().numpy(), t.std(0).clamp_min(1e-3).cpu().numpy()]
    m.set_normalization(*norm)
    grad, loss = m.gradient(feat, tgt)
    w16 = m.params.astype(np.float16).astype(np.float64)   # the kernels run on fp16 weights
    rl, rg = mlp_ref.loss_and_grad(w16, feat.cpu().numpy(), tgt.cpu().numpy(),
                                   *[np.asarray(a, np.float32).astype(np.float64) for a in norm])
    assert abs(loss - rl) <= 2e-2 * abs(rl)
    assert np.linalg.norm(grad - rg) <= 2e-2 * np.linalg.norm(rg)
    big = np.abs(rg) > 1e-2 * np.abs(rg).max()
    assert np.all(np.abs(grad[big] - rg[big]) <= 2e-2 * np.abs(rg[big]) + 1e-4 * np.abs(rg).max())


@pytest.mark.gpu
def test_training_learns_work_counts(c2small):
    from paper_2206_13574_gb300 import costmodel
    g, qs, graph = c2small
    m = gw.CostModel(graph, seed=5)
    eng = gw.Engine(graph)
    feat, tgt, _ = costmodel.collect(m, eng, qs.subset(np.arange(400)))
    losses = costmodel.fit(m, feat, tgt, steps=800, batch=256, lr=3e-3)
    assert losses[-50:].mean() < 0.5 * losses[:20].mean()
    tf, tt, _ = costmodel.collect(m, eng, qs.subset(np.arange(400, 600)))
    pred = m.predict(tf).cpu().numpy()
    r2 = costmodel.r2(pred, tt.cpu().numpy())
    assert r2[0] > 0.6 and r2[3] > 0.6, r2         # distance and work on held-out queries
    # the host evaluation (serving admission: host features, fp32 forward) agrees with
    # the device's (fp16 weights and activations) on held-out queries
    held = qs.subset(np.arange(400, 600))
    pall = m.predict(m.features(gw.DeviceBatch(held))).cpu().numpy()
    for i in range(0, 200, 10):
        h = m.predict_host(held.query(i), int(held.v_s[i]), int(held.v_e[i]))
        assert np.all(np.abs(h - pall[i]) <= 0.05 + 0.02 * np.abs(pall[i])), (i, h, pall[i])
    # the trained model through a file (gwfa_model_save / gwfa_model_load) predicts the same
    import tempfile
    path = os.path.join(tempfile.mkdtemp(), "model.bin")
    m.save(path)
    m2 = gw.CostModel(graph, seed=99)
    m2.load(path)
    assert np.array_equal(m2.params, m.params)
    assert all(np.array_equal(a, b) for a, b in zip(m2.norm, m.norm))
    assert np.array_equal(m2.predict(tf).cpu().numpy(), pred)
    with open(path, "r+b") as f:   # a damaged tag is refused
        f.write(b"X")
    with pytest.raises(gw.GwfaError):
        m2.load(path)


@pytest.mark.gpu
def test_learned_schedule_keeps_results_and_avoids_overflow_reruns(c2small):
    """Same results under the learned plan; fewer queries overflow tier 0 and run twice."""
    from paper_2206_13574_gb300 import costmodel
    g, qs, graph = c2small
    m = gw.CostModel(graph, seed=5)
    cfg = gw.default_config(graph)
    cfg.tiers[0].log2_tiles = 12             # small tier-0 slabs: overflow is common
    cfg.wide.ctas = 64
    cfg.wide.log2_tiles = 17
    eng = gw.Engine(graph, config=cfg)
    feat, tgt, _ = costmodel.collect(m, eng, qs.subset(np.arange(400)))
    costmodel.fit(m, feat, tgt, steps=800, batch=256, lr=3e-3)
    test = qs.subset(np.arange(400, 600))
    b = gw.DeviceBatch(test)
    b.run(eng)
    plain = b.results()
    plain_retries = int(eng.last_retries()[0])
    order, n_huge, n_wide = costmodel.plan(m, b, eng)
    assert n_huge == 0                       # no huge class in this engine
    b2 = gw.DeviceBatch(test, order=order)
    b2.run(eng, n_wide=n_wide)
    learned = b2.results()
    learned_retries = int(eng.last_retries()[0])
    for f in ("status", "edit_distance", "cells", "visited", "peak_frontier"):
        assert np.array_equal(plain[f], learned[f]), f
    assert plain_retries > 0
    assert learned_retries < plain_retries, (learned_retries, plain_retries, n_wide)


def test_lpt_packing_and_wide_class_sizing():
    """Host side of the plan: longest-first packing onto a work queue, and a large-slab
    class that gets one CTA per heavy query when those queries are the critical path."""
    from paper_2206_13574_gb300 import costmodel as cm
    assert cm.lpt_max_load([5, 4, 3, 3, 2], 2) == 9
    assert cm.lpt_max_load([1] * 10, 5) == 2
    assert cm.lpt_max_load([7], 3) == 7

    def pred_of(times):
        p = np.zeros((len(times), 4), np.float32)
        p[:, 0] = -1e-3                 # predicted distance ~0: time ~ cells without coefficients
        p[:, 3] = np.log1p(times)
        return p

    # 24 queries each as long as the whole batch would take: one CTA each
    t = np.concatenate([np.full(24, 100.0), np.ones(10000)])
    p = pred_of(t)
    order = np.argsort(-t, kind="stable")
    assert cm.wide_ctas(p, order, 24, 608) == 24
    # heavy but short next to the batch: the time share is enough
    t = np.concatenate([np.full(200, 5.0), np.ones(100000)])
    p = pred_of(t)
    order = np.argsort(-t, kind="stable")
    c = cm.wide_ctas(p, order, 200, 608)
    assert c < 200 and c >= round(608 * 1000 / 101000)
