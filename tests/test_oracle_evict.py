"""Pins of the memory-bounded H~ in the CPU oracle (with pruning, Alg. 4): entries
outside Q that lag a_max by evict_lag or more are removed every evict_every scores.
An evicted diagonal may come back, so the work changes, but every offset is still a
realised alignment: the distance is never below the exact one; a lag larger than
every a changes nothing; and fewer entries are held at the end."""
import pytest

import oracle
from paper_2206_13574_gb300 import synth

KEYS = ("distance", "is_upper_bound", "n_scores", "cells", "peak", "visited", "pruned", "spills")


@pytest.fixture(scope="module")
def c3():
    return synth.make_config(3, n_queries=4, backbone=200_000)


def test_huge_lag_changes_nothing(c3):
    g, qs = c3
    for i in range(len(qs)):
        args = (g, qs.query(i), int(qs.v_s[i]), int(qs.v_e[i]))
        a = oracle.gwfa(*args, a_diff=300)
        b = oracle.gwfa(*args, a_diff=300, evict_lag=10 ** 9, evict_every=8)
        assert {k: a[k] for k in KEYS} == {k: b[k] for k in KEYS} and b["evicted"] == 0


def test_bounded_memory(c3):
    g, qs = c3
    for i in range(2):
        args = (g, qs.query(i), int(qs.v_s[i]), int(qs.v_e[i]))
        free = oracle.gwfa(*args, a_diff=300)
        for lag, every in ((300, 16), (1500, 64)):
            b = oracle.gwfa(*args, a_diff=300, evict_lag=lag, evict_every=every)
            assert b["distance"] > 0 and b["evicted"] > 0
            # entries held at the end: insertions minus evictions
            assert b["visited"] - b["evicted"] < free["visited"]


def test_tiny_graphs_upper_bound():
    """The distance with eviction is never below the exact (Eq. 1) distance."""
    total = 0
    for t in range(200):
        r = synth.Rng(606, t)
        nv = r.one_int(1, 7)
        g = synth.random_small_graph(r, nv, 6, 0.3, t % 2 == 1)
        q = bytes(synth._ACGT[r.codes(r.one_int(0, 30))])
        d = oracle.dp_distance(g, q, 0, nv - 1)
        if d < 0:
            continue
        for lag in (1, 3, 8):
            s = oracle.gwfa(g, q, 0, nv - 1, a_diff=4, evict_lag=lag, evict_every=1)
            assert s["distance"] >= d, (t, lag, s, d)
            total += s["evicted"]
    assert total > 100


def test_rejects_bad_arguments():
    g = synth.Graph.from_lists([b"ACGT"], [])
    assert oracle.gwfa(g, b"ACG", 0, 0, evict_lag=5, evict_every=1)["distance"] == -1          # needs pruning
    assert oracle.gwfa(g, b"ACG", 0, 0, a_diff=5, evict_lag=5, evict_every=0)["distance"] == -1


PLANTED = ("GWFA_ORACLE_PLANT_EVICT_LE", "GWFA_ORACLE_PLANT_EVICT_OLDQ", "GWFA_ORACLE_PLANT_EVICT_BEFORE")


@pytest.mark.parametrize("plant", PLANTED)
def test_planted_eviction_mistakes_fail_the_hand_traces(plant, monkeypatch):
    """The two hand-traced eviction cases (tests/golden/handtrace.json) pin the rule:
    a planted mistake in the oracle -- keeping an entry that lags by exactly
    evict_lag, keeping by the Q that GwfExtend left instead of the new Q, or evicting
    before GwfExpand -- changes a traced counter on each of them (on the second, a
    counter other than `evicted`: the spill no longer re-inserts the diagonal)."""
    import json
    import os
    cases = [c for c in json.load(open(os.path.join(os.path.dirname(__file__), "golden", "handtrace.json")))["cases"]
             if c.get("evict_lag")]
    assert len(cases) >= 2
    monkeypatch.setenv(plant, "1")
    for c in cases:
        g = synth.Graph.from_lists(c["labels"], [tuple(a) for a in c["arcs"]])
        s = oracle.gwfa(g, c["q"].encode(), c["vs"], c["ve"], c["a_diff"], evict_lag=c["evict_lag"],
                        evict_every=c["evict_every"])
        changed = [k for k, v in c["expect"].items() if s[k] != v]
        assert changed, (plant, c["name"])
        if c["name"] == "evict_then_respill":
            assert set(changed) - {"evicted"}, (plant, changed)
