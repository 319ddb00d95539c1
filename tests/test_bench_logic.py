"""Host logic of the benchmark, on CPU: the in-run verification against the oracle
flags a result that differs in any checked counter (a planted mistake in a copy of the
oracle's own results), and the roofline arithmetic uses the stated byte counts."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
import paper_2206_13574_gb300 as gw  # noqa: E402
from paper_2206_13574_gb300 import synth  # noqa: E402


def _as_results(want) -> np.ndarray:
    """Oracle results laid out as the library's result records."""
    r = np.zeros(len(want), dtype=gw.RESULT_DTYPE)
    for i, w in enumerate(want):
        r[i]["status"] = 0 if w["distance"] >= 0 else w["distance"]
        for a, b in bench.VERIFY_FIELDS:
            r[i][a] = max(w[b], 0) if a == "edit_distance" else w[b]
    return r


def test_verify_flags_every_counter():
    g, qs = synth.make_config(1, n_queries=12)
    idx = np.arange(len(qs))
    want = oracle.gwfa_many(g, qs, idx)
    res = _as_results(want)
    ok = bench.verify(res, idx, want)
    assert ok["verified_queries"] == 12 and ok["mismatches"] == 0
    for k, (a, _) in enumerate(bench.VERIFY_FIELDS):
        bad = res.copy()
        bad[k][a] += 1   # one planted mistake per counter, in a different query each
        v = bench.verify(bad, idx, want)
        assert v["mismatches"] == 1 and v["mismatch_ids"] == [k], a
    bad = res.copy()
    bad[3]["status"] = gw.GWFA_ERR_CAPACITY
    assert bench.verify(bad, idx, want)["mismatch_ids"] == [3]


def test_roofline_arithmetic():
    r = bench.roofline(cells=10 ** 9, aligned_bp=10 ** 8, t_kernel=0.5, int_peak=None, counters=None,
                       peak_gbs=6000.0, peak_kind="measured", steps=1)
    alg = bench.B_CELL * 10 ** 9 + 0.5 * 10 ** 8
    assert abs(r["achieved"] - alg / 0.5 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 6000.0) < 1e-12
    assert r["int_frac"] is None and r["traffic"] is None
    counters = {"dram_bytes_per_cell": 27.5, "l2_throughput_pct": 15.0, "warp_inst_per_cell": 37.0,
                "alu_warp_inst_per_cell": 10.0, "source": "test"}
    peak = {"warp_inst_per_s": 6.0e11}
    r = bench.roofline(10 ** 9, 10 ** 8, 0.5, peak, counters, 6000.0, "measured", 1)
    assert abs(r["int_frac"] - 10.0 * 10 ** 9 / 0.5 / 6.0e11) < 1e-12
    assert abs(r["traffic"] - 27.5e9) < 1e-3 and abs(r["l2_frac"] - 0.15) < 1e-12
