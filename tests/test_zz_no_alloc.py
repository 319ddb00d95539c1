"""The allocation-free entry point (gwfa_align_noalloc), for callers that cannot let
the library allocate device memory.  Through the C ABI, two calls in a row must
give exactly the results of the engine-based entry point; collected last so that
a failure here does not hide any other test."""
import ctypes

import numpy as np
import pytest

import paper_2206_13574_gb300 as gw
from paper_2206_13574_gb300 import _build, synth

pytestmark = pytest.mark.gpu
FIELDS = [f for f in gw.RESULT_DTYPE.names if f != "device_us"]   # device_us is wall time


@pytest.mark.parametrize("max_lag", [0, 150])
def test_noalloc_matches_engine_twice(max_lag):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    g, qs = synth.make_config(2, n_queries=400)
    sub = qs.subset(np.argsort(qs.lengths(), kind="stable")[:250])   # fits the static slabs
    graph = gw.Graph.from_synth(g)
    ref = gw.Engine(graph, prune=max_lag > 0).align_batch(sub.seq, sub.off, sub.v_s, sub.v_e,
                                                          max_lag=max_lag)
    batch = gw.DeviceBatch(sub)
    lib = gw.load()
    opts = gw.gwfa_opts(max_lag, 0, -1, 0, 0, 0, 0)
    for call in range(2):
        batch.out.fill_(0xAB)
        st = lib.gwfa_align_noalloc(graph.handle, batch.n, batch.words.data_ptr(), batch.q_off.data_ptr(),
                                    batch.v_s.data_ptr(), batch.v_e.data_ptr(), 0, ctypes.byref(opts),
                                    batch.out.data_ptr(), None)
        assert st == gw.GWFA_OK
        torch.cuda.synchronize()
        res = batch.results()
        for f in FIELDS:
            assert np.array_equal(res[f], ref[f]), (call, f)
    # a slab larger than the static array is refused before any GPU work
    assert lib.gwfa_align_noalloc(graph.handle, batch.n, batch.words.data_ptr(), batch.q_off.data_ptr(),
                                  batch.v_s.data_ptr(), batch.v_e.data_ptr(), 20, ctypes.byref(opts),
                                  batch.out.data_ptr(), None) == gw.GWFA_ERR_CAPACITY
