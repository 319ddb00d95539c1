"""The allocation-free entry point (gwfa_align_noalloc).

Some callers cannot let the library allocate device memory: code running inside a
custom device allocator (allocating from there can deadlock or recurse), processes
whose memory another framework reserved up front, and loops that cannot pay for
cudaMalloc's implicit synchronisation.  gwfa_align_noalloc serves them from a fixed
array inside the library.  Through the C ABI, two calls in a row must give exactly
the results of the engine-based entry point (and of the oracle), reject a query the
packing found invalid, and report a query too large for its slab as a capacity
error while its neighbours stay exact.  Collected last so that a failure here does
not hide any other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2206_13574_gb300 as gw
from paper_2206_13574_gb300 import _build, synth

pytestmark = pytest.mark.gpu
FIELDS = [f for f in gw.RESULT_DTYPE.names if f != "device_us"]   # device_us is wall time


def _call(lib, graph, batch, log2_tiles, opts):
    return lib.gwfa_align_noalloc(graph.handle, batch.n, batch.words.data_ptr(), batch.q_off.data_ptr(),
                                  batch.v_s.data_ptr(), batch.v_e.data_ptr(), batch.status.data_ptr(),
                                  log2_tiles, ctypes.byref(opts), batch.out.data_ptr(), None)


def _with_invalid_base(qs, i):
    """A copy of the batch whose query i carries an N (not A/C/G/T) in its middle."""
    seq = qs.seq.copy()
    seq[int(qs.off[i]) + int(qs.off[i + 1] - qs.off[i]) // 2] = ord("N")
    return synth.Queries(seq=seq, off=qs.off.copy(), v_s=qs.v_s.copy(), v_e=qs.v_e.copy(),
                         edits=qs.edits.copy(), divergence=qs.divergence.copy())


@pytest.mark.parametrize("max_lag", [0, 150])
def test_noalloc_matches_engine_twice(max_lag):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    g, qs = synth.make_config(2, n_queries=400)
    sub = qs.subset(np.argsort(qs.lengths(), kind="stable")[:250])   # fits the static slabs
    bad = 17
    sub = _with_invalid_base(sub, bad)
    graph = gw.Graph.from_synth(g)
    ref = gw.Engine(graph, prune=max_lag > 0).align_batch(sub.seq, sub.off, sub.v_s, sub.v_e,
                                                          max_lag=max_lag)
    assert ref["status"][bad] == gw.GWFA_ERR_INVALID
    batch = gw.DeviceBatch(sub)
    lib = gw.load()
    opts = gw.gwfa_opts(max_lag, 0, -1, 0, 0, 0, 0)
    for call in range(2):
        batch.out.fill_(0xAB)
        assert _call(lib, graph, batch, 0, opts) == gw.GWFA_OK
        torch.cuda.synchronize()
        res = batch.results()
        for f in FIELDS:
            assert np.array_equal(res[f], ref[f]), (call, f)
        assert res["status"][bad] == gw.GWFA_ERR_INVALID
    # a few results straight against the oracle (Alg. 1-4 on the CPU)
    for i in (0, 60, 249):
        w = oracle.gwfa(g, sub.query(i), int(sub.v_s[i]), int(sub.v_e[i]), a_diff=max_lag)
        got = (int(res["edit_distance"][i]), int(res["cells"][i]), int(res["peak_frontier"][i]),
               int(res["visited"][i]), int(res["pruned"][i]))
        assert got == (w["distance"], w["cells"], w["peak"], w["visited"], w["pruned"]), i
    # a slab larger than the static array is refused before any GPU work, and a
    # log2_tiles outside the supported range is an argument error
    assert _call(lib, graph, batch, 20, opts) == gw.GWFA_ERR_CAPACITY
    assert _call(lib, graph, batch, 7, opts) == gw.GWFA_ERR_INVALID
    assert _call(lib, graph, batch, 25, opts) == gw.GWFA_ERR_INVALID


def test_noalloc_overflow_is_a_capacity_error():
    """With 2^10-tile slabs (a query may claim 768 tiles), a query whose oracle
    visits more than 8 x 768 diagonals cannot fit (a tile holds 8), and one that
    visits at most 768 always fits (every claimed tile holds a visited diagonal):
    the first ends GWFA_ERR_CAPACITY, there being no overflow tier, and the others
    equal the engine's results, on two calls in a row."""
    import torch
    _build.build()
    g, qs = synth.make_config(2, n_queries=400)
    by_len = np.argsort(qs.lengths(), kind="stable")
    cand = np.concatenate([by_len[:120], by_len[-40:]])
    ora = oracle.gwfa_many(g, qs, cand)
    vis = np.array([w["visited"] for w in ora])
    fits = cand[vis <= 768][:60]
    big = cand[vis > 8 * 768][:2]
    assert len(fits) >= 20 and len(big) >= 1
    pick = np.concatenate([fits[:30], big, fits[30:]])
    sub = qs.subset(pick)
    big_pos = np.arange(30, 30 + len(big))
    graph = gw.Graph.from_synth(g)
    ref = gw.Engine(graph).align_batch(sub.seq, sub.off, sub.v_s, sub.v_e)
    batch = gw.DeviceBatch(sub)
    lib = gw.load()
    opts = gw.gwfa_opts(0, 0, -1, 0, 0, 0, 0)
    rest = np.setdiff1d(np.arange(len(pick)), big_pos)
    for call in range(2):
        batch.out.fill_(0xAB)
        assert _call(lib, graph, batch, 10, opts) == gw.GWFA_OK
        torch.cuda.synchronize()
        res = batch.results()
        assert np.all(res["status"][big_pos] == gw.GWFA_ERR_CAPACITY), call
        for f in FIELDS:
            assert np.array_equal(res[f][rest], ref[f][rest]), (call, f)
    assert np.all(ref["status"] == 0)
