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
