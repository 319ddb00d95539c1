"""Base-level alignment along the traceback walk (the pairwise step the paper's
discussion, Sec. 4, adds after Alg. 6), on the GPU: every CIGAR must be a valid
alignment of the query to the sequence its walk spells, with exactly the Gwfa edit
distance of edits, and that cost must equal the oracle's Levenshtein distance of
the two sequences."""
import numpy as np
import pytest

import oracle
import paper_2206_13574_gb300 as gw
from paper_2206_13574_gb300 import _build, synth
from cigar_check import apply_cigar

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    oracle.build()


def traceback_batch(graph, qs, path_cap=4096, ends=0):
    """Exact distances and walks of a batch (traceback engine, max_lag 0)."""
    import torch
    eng = gw.Engine(graph, prune=True)
    paths = torch.zeros(len(qs) * path_cap, dtype=torch.int32, device="cuda")
    plen = torch.zeros(len(qs), dtype=torch.int32, device="cuda")
    eng.set_paths(paths.data_ptr(), path_cap, plen.data_ptr())
    b = gw.DeviceBatch(qs)
    b.run(eng, traceback=True, ends=ends)
    torch.cuda.synchronize()
    return eng, b, paths, plen


def cigars(graph, b, paths, plen, path_cap=4096, cigar_cap=1024, ends=0, **kw):
    import torch
    cg = gw.Cigar(graph, **kw)
    ops, out = cg.run(b, paths, plen, path_cap, cigar_cap, ends=ends)
    torch.cuda.synchronize()
    res = out.cpu().numpy().view(gw.CIGAR_RESULT_DTYPE)
    cg.close()
    return ops.view(b.n, cigar_cap).cpu().numpy().view(np.uint32), res


def queries(seqs, vs, ve) -> synth.Queries:
    off = np.zeros(len(seqs) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(x) for x in seqs])
    return synth.Queries(seq=np.frombuffer(b"".join(seqs), dtype=np.uint8).copy(), off=off,
                         v_s=np.asarray(vs, np.uint32), v_e=np.asarray(ve, np.uint32),
                         edits=np.zeros(len(seqs), np.int64), divergence=np.zeros(len(seqs)))


def spelled(g, walk) -> bytes:
    return b"".join(g.label(int(v)) for v in walk)


def check_batch(g, qs, res, P, L, ops, cr, lev_idx=()):
    for i in range(len(qs)):
        assert res[i]["status"] == 0
        t = spelled(g, P[i, :L[i]])
        r = cr[i]
        assert r["status"] == 0, (i, r)
        assert r["walk_len"] == len(t)
        assert r["cost"] == res[i]["edit_distance"]
        assert apply_cigar(qs.query(i), t, ops[i, :r["n_ops"]]) == r["cost"]
    for i in lev_idx:
        assert oracle.levenshtein(qs.query(i), spelled(g, P[i, :L[i]])) == cr[i]["cost"]


def test_config1_all_queries():
    g, qs = synth.make_config(1)
    graph = gw.Graph.from_synth(g)
    eng, b, paths, plen = traceback_batch(graph, qs)
    res = b.results()
    ops, cr = cigars(graph, b, paths, plen)
    P = paths.view(len(qs), -1).cpu().numpy()
    L = plen.cpu().numpy()
    check_batch(g, qs, res, P, L, ops, cr, lev_idx=range(len(qs)))


def test_config2_batch():
    g, qs = synth.make_config(2, n_queries=300)
    graph = gw.Graph.from_synth(g)
    eng, b, paths, plen = traceback_batch(graph, qs)
    res = b.results()
    ops, cr = cigars(graph, b, paths, plen, cigar_cap=4096, workspace_bytes=32 << 20)
    P = paths.view(len(qs), -1).cpu().numpy()
    L = plen.cpu().numpy()
    short = np.argsort(qs.lengths())[:25]
    check_batch(g, qs, res, P, L, ops, cr, lev_idx=short)


def test_tiny_cyclic_graphs():
    """Walks through cycles revisit vertices; the spelled sequence repeats labels."""
    for t in range(12):
        rr = synth.Rng(91, t)
        nv = rr.one_int(2, 7)
        g2 = synth.random_small_graph(rr, nv, 12, 0.35, True)
        qs = queries([bytes(synth._ACGT[rr.codes(rr.one_int(1, 40))]) for _ in range(6)],
                     [0] * 6, [nv - 1] * 6)
        graph = gw.Graph.from_synth(g2)
        eng, b, paths, plen = traceback_batch(graph, qs, path_cap=512)
        res = b.results()
        ops, cr = cigars(graph, b, paths, plen, path_cap=512, cigar_cap=256, ctas=3)
        P = paths.view(len(qs), -1).cpu().numpy()
        L = plen.cpu().numpy()
        for i in range(len(qs)):
            assert res[i]["edit_distance"] == oracle.dp_distance(g2, qs.query(i), 0, nv - 1)
        check_batch(g2, qs, res, P, L, ops, cr, lev_idx=range(len(qs)))
        eng.close()
        graph.close()


def test_capacity_limits_are_reported():
    g, qs = synth.make_config(2, n_queries=120)
    graph = gw.Graph.from_synth(g)
    eng, b, paths, plen = traceback_batch(graph, qs)
    res = b.results()
    full_ops, full = cigars(graph, b, paths, plen, cigar_cap=4096, workspace_bytes=32 << 20)
    # a small workspace: queries with large distances do not fit
    ops, small = cigars(graph, b, paths, plen, cigar_cap=4096, workspace_bytes=256 << 10)
    d = res["edit_distance"].astype(np.int64)
    m = full["walk_len"].astype(np.int64)
    c = np.ceil(np.sqrt(d + 1)).astype(np.int64)   # checkpoint spacing
    c = np.where(c * c < d + 1, c + 1, c)
    need = ((m // 16 + 2) * 4 + 15) // 16 * 16 + (d // c + c + 2) * (2 * d + 1) * 4
    fits = need <= (256 << 10)
    assert fits.any() and (~fits).any()
    assert np.all(small["status"][~fits] == gw.GWFA_ERR_CAPACITY)
    assert np.all(small["status"][fits] == 0)
    for i in np.nonzero(fits)[0]:
        assert np.array_equal(ops[i, :small[i]["n_ops"]], full_ops[i, :full[i]["n_ops"]])
    # too few operation slots: the count is still reported
    ops, few = cigars(graph, b, paths, plen, cigar_cap=4, workspace_bytes=32 << 20)
    over = full["n_ops"] > 4
    assert over.any()
    assert np.all(few["status"][over] == gw.GWFA_ERR_CAPACITY)
    assert np.array_equal(few["n_ops"], full["n_ops"])


def test_failed_queries_are_not_run():
    g, qs = synth.make_config(1, n_queries=8)
    qs.v_e[3] = 10 ** 6   # out of range: the alignment itself fails
    graph = gw.Graph.from_synth(g)
    eng, b, paths, plen = traceback_batch(graph, qs)
    res = b.results()
    assert res[3]["status"] != 0
    ops, cr = cigars(graph, b, paths, plen)
    assert cr[3]["status"] == gw.GWFA_ERR_NOT_RUN
    assert np.all(cr["status"][np.arange(8) != 3] == 0)


@pytest.mark.parametrize("ends", [1, 2, 3, 4, 5])   # FREE_START, FREE_END, both, EXTEND, EXTEND|FREE_START
def test_formulation_variants(ends):
    """With free walk ends the CIGAR aligns the whole query to [walk_begin, walk_end)
    of sigma(w): the skipped prefix lies in the first vertex, the skipped suffix in the
    last one, and the cost is the variant distance."""
    g, qs0 = synth.make_config(1)
    r = synth.Rng(ends, 3)
    seqs = []
    for i in range(len(qs0)):   # cut a few bases from both ends so that free ends matter
        q = qs0.query(i)
        a = r.one_int(0, min(len(g.label(int(qs0.v_s[i]))), 20))
        b = r.one_int(0, min(len(g.label(int(qs0.v_e[i]))), 20))
        seqs.append(q[a:len(q) - b])
    qs = queries(seqs, qs0.v_s, qs0.v_e)
    graph = gw.Graph.from_synth(g)
    eng, b, paths, plen = traceback_batch(graph, qs, ends=ends)
    res = b.results()
    ops, cr = cigars(graph, b, paths, plen, ends=ends)
    P = paths.view(len(qs), -1).cpu().numpy()
    L = plen.cpu().numpy()
    for i in range(len(qs)):
        assert res[i]["status"] == 0
        walk = P[i, :L[i]]
        t = spelled(g, walk)
        c = cr[i]
        assert c["status"] == 0, (i, c)
        assert c["cost"] == res[i]["edit_distance"] == oracle.dp_distance(
            g, qs.query(i), int(qs.v_s[i]), int(qs.v_e[i]), ends=ends)
        first, last = len(g.label(int(walk[0]))), len(g.label(int(walk[-1])))
        assert c["walk_begin"] <= (first if ends & 1 else 0)
        assert c["walk_end"] >= (len(t) - last if ends & 6 else len(t)) and c["walk_end"] <= len(t)
        assert apply_cigar(qs.query(i), t[c["walk_begin"]:c["walk_end"]], ops[i, :c["n_ops"]]) == c["cost"]


def test_large_distances_config4_style():
    """Distances of thousands (the large workload's 5-10% divergence on tens of kb):
    the checkpointed backtrace keeps about 2 sqrt(d) wavefronts, so these fit the
    default 32 MiB per CTA; every CIGAR is valid, costs the Gwfa distance, and equals
    the oracle's Levenshtein distance of the query and the spelled walk."""
    from concurrent.futures import ThreadPoolExecutor
    import os
    g, q0 = synth.make_config(4, n_queries=600, backbone=3_000_000)
    L0 = q0.lengths()
    mid = np.nonzero((q0.divergence > 0.05) & (L0 > 15_000) & (L0 < 45_000))[0][:5]
    far = np.nonzero((q0.divergence > 0.08) & (L0 > 60_000) & (L0 < 100_000))[0][:1]   # d ~ 6,000
    pick = np.concatenate([mid, far])
    assert len(pick) >= 5
    qs = q0.subset(pick)
    graph = gw.Graph.from_synth(g)
    cap = 16384
    eng, b, paths, plen = traceback_batch(graph, qs, path_cap=cap)
    res = b.results()
    assert res["edit_distance"].max() > 5000
    ops, cr = cigars(graph, b, paths, plen, path_cap=cap, cigar_cap=32768)
    P = paths.view(len(qs), -1).cpu().numpy()
    L = plen.cpu().numpy()
    check_batch(g, qs, res, P, L, ops, cr)
    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        lev = list(ex.map(lambda i: oracle.levenshtein(qs.query(i), spelled(g, P[i, :L[i]])), range(len(qs))))
    assert lev == [int(x) for x in cr["cost"]]
