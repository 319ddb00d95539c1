"""Pins of the formulation variants (Sec. 2.1: a walk that may start or end inside
its end vertices, and extension without an end vertex) in the CPU oracle, against
brute-force enumeration of walks and of the prefixes / suffixes they may skip, and
against closed forms; then the variant Gwfa (Alg. 1-3 with the variant start and
end test) against the variant DP."""
import pytest

import oracle
from oracle import EXTEND, FREE_END, FREE_START, brute
from paper_2206_13574_gb300 import synth

VARIANTS = [FREE_START, FREE_END, FREE_START | FREE_END, EXTEND, EXTEND | FREE_START]


def _lists(g):
    labels = [g.label(v) for v in range(g.n_vertices)]
    arcs = list(zip(g.arc_src.tolist(), g.arc_dst.tolist()))
    return labels, arcs


def _rand_q(r, n):
    return bytes(synth._ACGT[r.codes(n)])


@pytest.mark.parametrize("ends", VARIANTS)
@pytest.mark.parametrize("cyclic", [False, True])
def test_dp_variants_match_enumeration(ends, cyclic):
    bad = []
    for t in range(100):
        r = synth.Rng(2000 + ends * 7 + int(cyclic), t)
        nv = r.one_int(1, 6)
        g = synth.random_small_graph(r, nv, 4, 0.3, cyclic)
        labels, arcs = _lists(g)
        q = _rand_q(r, r.one_int(0, 7 if cyclic else 9))
        vs = r.one_int(0, nv - 1)
        ve = r.one_int(vs, nv - 1)
        want = brute.best_walk_distance_ends(labels, arcs, q, vs, ve, bool(ends & FREE_START),
                                             bool(ends & FREE_END), bool(ends & EXTEND))
        got = oracle.dp_distance(g, q, vs, ve, ends=ends)
        if want is None:
            assert got < 0
        elif got != want:
            bad.append((t, labels, arcs, q, vs, ve, want, got))
    assert not bad, bad[:3]


def test_closed_forms():
    r = synth.Rng(31, 0)
    for _ in range(100):
        lab = _rand_q(r, r.one_int(5, 40))
        a = r.one_int(0, len(lab) - 1)
        b = r.one_int(a, len(lab))
        g = synth.Graph.from_lists([lab], [])
        # a piece of the label: 0 with both ends free, the skipped length with one
        assert oracle.dp_distance(g, lab[a:b], 0, 0, ends=FREE_START | FREE_END) == 0
        assert oracle.dp_distance(g, lab[a:], 0, 0, ends=FREE_START) == 0
        assert oracle.dp_distance(g, lab[:b], 0, 0, ends=FREE_END) == 0
        assert oracle.dp_distance(g, lab[:b], 0, 0, ends=EXTEND) == 0
        assert oracle.dp_distance(g, lab[a:b], 0, 0) == len(lab) - (b - a)
        # both ends free on one vertex = the best substring match
        q = _rand_q(r, r.one_int(0, 12))
        want = min(brute.levenshtein_py(lab[x:y], q) for x in range(len(lab) + 1)
                   for y in range(x, len(lab) + 1))
        assert oracle.dp_distance(g, q, 0, 0, ends=FREE_START | FREE_END) == want


def test_variants_only_relax():
    """Freeing an end can only lower the distance; extension may end anywhere,
    v_e's cells included."""
    for t in range(150):
        r = synth.Rng(77, t)
        nv = r.one_int(1, 7)
        g = synth.random_small_graph(r, nv, 6, 0.3, t % 2 == 1)
        q = _rand_q(r, r.one_int(0, 14))
        vs, ve = 0, nv - 1
        d = {e: oracle.dp_distance(g, q, vs, ve, ends=e) for e in [0] + VARIANTS}
        if d[0] < 0:
            continue
        assert d[FREE_START] <= d[0] and d[FREE_END] <= d[0]
        assert d[FREE_START | FREE_END] <= min(d[FREE_START], d[FREE_END])
        assert d[EXTEND] <= d[FREE_END]
        assert d[EXTEND | FREE_START] <= min(d[EXTEND], d[FREE_START | FREE_END])


@pytest.mark.parametrize("ends", VARIANTS)
@pytest.mark.parametrize("cyclic", [False, True])
def test_gwfa_variants_equal_dp(ends, cyclic):
    for t in range(150):
        r = synth.Rng(5000 + ends * 3 + int(cyclic), t)
        nv = r.one_int(1, 7)
        g = synth.random_small_graph(r, nv, 5, 0.3, cyclic)
        q = _rand_q(r, r.one_int(0, 14))
        vs = r.one_int(0, nv - 1)
        ve = r.one_int(vs, nv - 1)
        d = oracle.dp_distance(g, q, vs, ve, ends=ends)
        s = oracle.gwfa(g, q, vs, ve, ends=ends)
        assert s["distance"] == d, (t, ends, d, s)
        if d >= 0:
            assert s["n_scores"] == d + 1


def test_gwfa_variants_config1_sample():
    g, qs = synth.make_config(1)
    for ends in VARIANTS:
        for i in range(0, len(qs), 9):
            q, vs, ve = qs.query(i), int(qs.v_s[i]), int(qs.v_e[i])
            assert oracle.gwfa(g, q, vs, ve, ends=ends)["distance"] == oracle.dp_distance(g, q, vs, ve, ends=ends)


def test_variants_reject_pruning_and_bad_flags():
    g = synth.Graph.from_lists([b"ACGT"], [])
    assert oracle.gwfa(g, b"ACG", 0, 0, a_diff=10, ends=FREE_END)["distance"] == -1
    assert oracle.dp_distance(g, b"ACG", 0, 0, ends=8) == -1
