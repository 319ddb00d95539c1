"""Pin of the walk-base tie rule of the pruned oracle (reading: a diagonal absent when
spilled into takes the largest base among the spills of the same FIFO generation).

The rule exists so that the result does not depend on the order in which the FIFO
queue meets the spills -- the property every parallel execution relies on.  Reversing
or shuffling the arc lists changes that order; the pruned results (distance and every
work count) must not change.  The same check against a planted mistake (first spill
wins, switched on in the oracle for this test only) must find graphs where the order
does change the result, so the check has teeth."""
import os

import oracle
from paper_2206_13574_gb300 import synth

PLANT = "GWFA_ORACLE_PLANT_FIRST_TIE"


def _cases(n):
    for t in range(n):
        r = synth.Rng(808, t)
        nv = r.one_int(3, 8)
        g = synth.random_small_graph(r, nv, 4, 0.45, t % 2 == 1)
        labels = [g.label(v) for v in range(g.n_vertices)]
        arcs = list(zip(g.arc_src.tolist(), g.arc_dst.tolist()))
        order = sorted(range(len(arcs)), key=lambda a: r.one_int(0, 1 << 30))
        g2 = synth.Graph.from_lists(labels, [arcs[a] for a in order])
        g3 = synth.Graph.from_lists(labels, arcs[::-1])
        q = bytes(synth._ACGT[r.codes(r.one_int(4, 24))])
        yield g, g2, g3, q, nv, r.one_int(1, 6)


def test_pruned_results_do_not_depend_on_arc_order():
    planted_changes = 0
    for g, g2, g3, q, nv, a_diff in _cases(600):
        a = oracle.gwfa(g, q, 0, nv - 1, a_diff=a_diff)
        assert a == oracle.gwfa(g2, q, 0, nv - 1, a_diff=a_diff), (q, a_diff)
        assert a == oracle.gwfa(g3, q, 0, nv - 1, a_diff=a_diff), (q, a_diff)
        os.environ[PLANT] = "1"
        try:
            b = [oracle.gwfa(x, q, 0, nv - 1, a_diff=a_diff) for x in (g, g2, g3)]
        finally:
            del os.environ[PLANT]
        planted_changes += int(not (b[0] == b[1] == b[2]))
    assert planted_changes > 0
