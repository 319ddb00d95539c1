"""Pins of the CPU oracle against things other than itself (no GPU needed).

* Eq. 1 DP (oracle_dp) vs explicit walk enumeration (brute.py) on tiny DAGs and
  tiny cyclic graphs; vs Levenshtein on single-vertex and chain graphs (Sec. 2.2:
  a chain of vertices is the concatenated string); closed forms (error-free walk
  copies give 0; |q| = 0 gives the shortest spelled walk; the distance is at least
  the gap between |q| and every walk length, at most the number of injected edits).
* Alg. 1-3 (oracle_gwfa, exact) vs Eq. 1 (Gwfa is exact, Sec. 2.4), and its work
  counts vs hand traces (tests/golden/handtrace.json).
* Alg. 4 (pruned): upper bound of the exact distance (Sec. 2.5: pruning may miss
  the optimum), equal to exact mode with identical work when a_diff exceeds every
  a, and the hand traces.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2206_13574_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "handtrace.json")


def _lists(g):
    labels = [g.label(v) for v in range(g.n_vertices)]
    arcs = list(zip(g.arc_src.tolist(), g.arc_dst.tolist()))
    return labels, arcs


def _rand_q(r, n):
    return bytes(synth._ACGT[r.codes(n)])


# ---------------------------------------------------------------- Levenshtein


def test_levenshtein_closed_forms():
    assert oracle.levenshtein(b"", b"") == 0
    assert oracle.levenshtein(b"ACGT", b"") == 4
    assert oracle.levenshtein(b"", b"GATTACA") == 7
    assert oracle.levenshtein(b"GATTACA", b"GATTACA") == 0
    assert oracle.levenshtein(b"GATTACA", b"GATCACA") == 1      # one substitution
    assert oracle.levenshtein(b"GATTACA", b"GATACA") == 1       # one deletion
    assert oracle.levenshtein(b"GATTACA", b"GATTTACA") == 1     # one insertion
    assert oracle.levenshtein(b"AAAA", b"TTTT") == 4
    assert oracle.levenshtein(b"ACGTACGT", b"CGTACGTA") == 2    # shift by one = del + ins


def test_levenshtein_matches_python_and_axioms():
    r = synth.Rng(11, 0)
    for _ in range(200):
        x = _rand_q(r, r.one_int(0, 12))
        y = _rand_q(r, r.one_int(0, 12))
        z = _rand_q(r, r.one_int(0, 12))
        dxy = oracle.levenshtein(x, y)
        assert dxy == brute.levenshtein_py(x, y)
        assert dxy == oracle.levenshtein(y, x)
        assert abs(len(x) - len(y)) <= dxy <= max(len(x), len(y))
        assert oracle.levenshtein(x, z) <= dxy + oracle.levenshtein(y, z)


# ---------------------------------------------------------------- Eq. 1 DP


@pytest.mark.parametrize("cyclic", [False, True])
def test_dp_matches_walk_enumeration(cyclic):
    bad = []
    for t in range(300):
        r = synth.Rng(1234 + int(cyclic), t)
        nv = r.one_int(1, 7)
        g = synth.random_small_graph(r, nv, 4, 0.3, cyclic)
        labels, arcs = _lists(g)
        q = _rand_q(r, r.one_int(0, 10))
        vs = r.one_int(0, nv - 1)
        ve = r.one_int(vs, nv - 1)
        want = brute.best_walk_distance(labels, arcs, q, vs, ve)
        got = oracle.dp_distance(g, q, vs, ve)
        if want is None:
            assert got < 0
        elif got != want:
            bad.append((t, labels, arcs, q, vs, ve, want, got))
    assert not bad, bad[:3]


def test_dp_single_vertex_is_levenshtein():
    r = synth.Rng(5, 5)
    for _ in range(200):
        lab = _rand_q(r, r.one_int(1, 30))
        q = _rand_q(r, r.one_int(0, 30))
        g = synth.Graph.from_lists([lab], [])
        assert oracle.dp_distance(g, q, 0, 0) == brute.levenshtein_py(lab, q)


def test_dp_chain_is_concatenated_string():
    """Sec. 2.2: compacting a chain of vertices into one string keeps the recurrence."""
    r = synth.Rng(6, 6)
    for _ in range(100):
        s = _rand_q(r, r.one_int(1, 40))
        cuts = sorted(set(int(c) for c in r.integers(1, max(1, len(s) - 1), 4))) if len(s) > 1 else []
        pieces, p0 = [], 0
        for c in cuts + [len(s)]:
            if c > p0:
                pieces.append(s[p0:c])
                p0 = c
        g = synth.Graph.from_lists(pieces, [(i, i + 1) for i in range(len(pieces) - 1)])
        q = _rand_q(r, r.one_int(0, 40))
        assert oracle.dp_distance(g, q, 0, len(pieces) - 1) == brute.levenshtein_py(s, q)


def test_dp_empty_query_is_shortest_walk():
    for t in range(100):
        r = synth.Rng(77, t)
        nv = r.one_int(1, 8)
        g = synth.random_small_graph(r, nv, 5, 0.3, t % 2 == 1)
        labels, arcs = _lists(g)
        want = brute.shortest_spelled_walk(labels, arcs, 0, nv - 1)
        assert oracle.dp_distance(g, b"", 0, nv - 1) == want


def test_dp_error_free_and_injected_edit_bounds():
    g, qs = synth.make_config(1)
    dist = oracle.dp_many(g, qs, range(len(qs)))
    assert all(d <= e for d, e in zip(dist, qs.edits))        # d <= injected edits
    assert any(d > 0 for d in dist)
    # error-free copies of the same walks: distance 0
    c = synth.CONFIGS[1]
    clean = synth.make_queries(g, 30, 1, c["length"], lambda r: 0.0)
    assert all(d == 0 for d in oracle.dp_many(g, clean, range(len(clean))))


def test_dp_lower_bound_by_walk_lengths():
    """d >= min over s->e walks |n - len(walk)| (a DAG: walk lengths by a set DP)."""
    g, qs = synth.make_config(1, n_queries=20)
    lens = g.lengths()
    succ = {}
    for u, v in zip(g.arc_src.tolist(), g.arc_dst.tolist()):
        succ.setdefault(u, []).append(v)
    for i in range(len(qs)):
        vs, ve, n = int(qs.v_s[i]), int(qs.v_e[i]), int(qs.lengths()[i])
        reach = {vs: {int(lens[vs])}}
        for v in range(vs, ve + 1):          # ids are a topological order
            for u in succ.get(v, []):
                if u <= ve and v in reach:
                    reach.setdefault(u, set()).update(L + int(lens[u]) for L in reach[v])
        lb = min(abs(n - L) for L in reach[ve])
        assert oracle.dp_distance(g, qs.query(i), vs, ve) >= lb


def test_dp_rejects_bad_input():
    g = synth.Graph.from_lists(["ACGT", "GG"], [(0, 1)])
    assert oracle.dp_distance(g, b"ACGN", 0, 1) < 0            # not ACGT
    assert oracle.dp_distance(g, b"ACGT", 1, 0) == -4           # unreachable
    g2 = synth.Graph.from_lists(["ACGT", ""], [(0, 1)])
    assert oracle.dp_distance(g2, b"ACGT", 0, 0) < 0            # empty label


# ---------------------------------------------------------------- Alg. 1-4


@pytest.mark.parametrize("cyclic", [False, True])
def test_gwfa_exact_equals_dp_tiny(cyclic):
    for t in range(300):
        r = synth.Rng(4321 + int(cyclic), t)
        nv = r.one_int(1, 7)
        g = synth.random_small_graph(r, nv, 5, 0.3, cyclic)
        q = _rand_q(r, r.one_int(0, 14))
        vs = r.one_int(0, nv - 1)
        ve = r.one_int(vs, nv - 1)
        d = oracle.dp_distance(g, q, vs, ve)
        s = oracle.gwfa(g, q, vs, ve)
        assert s["distance"] == d, (t, d, s)
        if d >= 0:
            assert s["n_scores"] == d + 1
            assert s["peak"] <= s["cells"] and s["visited"] <= s["cells"]


def test_gwfa_exact_equals_dp_config1():
    g, qs = synth.make_config(1)
    dp = oracle.dp_many(g, qs, range(len(qs)))
    gw = oracle.gwfa_many(g, qs, range(len(qs)))
    assert [x["distance"] for x in gw] == dp


def test_gwfa_exact_equals_dp_config2_sample():
    g, qs = synth.make_config(2, n_queries=60)
    idx = np.argsort(qs.lengths())[:24]
    dp = oracle.dp_many(g, qs, idx)
    gw = oracle.gwfa_many(g, qs, idx)
    assert [x["distance"] for x in gw] == dp


def test_gwfa_exact_equals_dp_cyclic_config3_small():
    """Tandem-repeat loops (self arcs) on a short backbone, short queries."""
    g, _ = synth.make_config(3, n_queries=1, backbone=30000)
    c = synth.CONFIGS[3]
    qs = synth.make_queries(g, 12, 33, lambda r: 1500, c["div"], c["weights"], c["loops"])
    dp = oracle.dp_many(g, qs, range(len(qs)))
    gw = oracle.gwfa_many(g, qs, range(len(qs)))
    assert [x["distance"] for x in gw] == dp


def test_gwfa_handtraced_golden():
    cases = json.load(open(GOLDEN))["cases"]
    for c in cases:
        g = synth.Graph.from_lists(c["labels"], [tuple(a) for a in c["arcs"]])
        s = oracle.gwfa(g, c["q"].encode(), c["vs"], c["ve"], c["a_diff"],
                        evict_lag=c.get("evict_lag", 0), evict_every=c.get("evict_every", 0))
        for k, v in c["expect"].items():
            assert s[k] == v, (c["name"], k, s[k], v)
        if c["a_diff"] == 0:
            assert oracle.dp_distance(g, c["q"].encode(), c["vs"], c["ve"]) == c["expect"]["distance"]


def test_pruned_is_upper_bound_and_large_lag_is_exact():
    g, qs = synth.make_config(2, n_queries=40)
    idx = range(40)
    ex = oracle.gwfa_many(g, qs, idx)
    pr = oracle.gwfa_many(g, qs, idx, a_diff=200)
    big = oracle.gwfa_many(g, qs, idx, a_diff=10 ** 9)
    for e, p, b in zip(ex, pr, big):
        assert p["distance"] >= e["distance"]
        if p["is_upper_bound"] == 0:
            assert p["distance"] == e["distance"]
        assert b == e          # a_diff above every a: pruning never fires
    assert any(p["is_upper_bound"] for p in pr)


def test_gwfa_score_limit_and_unreachable():
    g = synth.Graph.from_lists(["ACGTACGT", "TT"], [(0, 1)])
    assert oracle.gwfa(g, b"TTTTTTTTTT", 0, 1, max_score=2)["distance"] == -8
    assert oracle.gwfa(g, b"ACGT", 1, 0)["distance"] == -4
