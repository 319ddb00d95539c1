"""Python binding of libgwfa.so (graph wavefront alignment on GB300).

Argument marshalling only: every step of the alignment runs in the library's
CUDA kernels.  Names follow the C ABI in include/gwfa.h.  PyTorch is used only
to hold device buffers and to pass the current CUDA stream.  There is no CPU
fallback: if libgwfa.so is missing or no GPU is usable, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgwfa.so")

GWFA_OK = 0
GWFA_PENDING = 1
GWFA_ERR_INVALID = -1
GWFA_ERR_OOM = -2
GWFA_ERR_CUDA = -3
GWFA_ERR_UNREACHABLE = -4
GWFA_ERR_EMPTY_FRONTIER = -5
GWFA_ERR_CAPACITY = -6
GWFA_ERR_TIMEOUT = -7
GWFA_ERR_SCORE_LIMIT = -8
GWFA_ERR_NOT_RUN = -9
GWFA_MAX_TIERS = 4

# numpy view of gwfa_result (64 bytes)
RESULT_DTYPE = np.dtype([("status", "<i4"), ("edit_distance", "<i4"), ("is_upper_bound", "<i4"),
                         ("n_scores", "<u4"), ("cells", "<u8"), ("visited", "<u8"),
                         ("peak_frontier", "<u4"), ("device_us", "<u4"), ("pruned", "<u8"),
                         ("spills", "<u8"), ("evicted", "<u8")])
assert RESULT_DTYPE.itemsize == 64

# numpy view of gwfa_cigar_result (24 bytes) and the CIGAR op codes (BAM's)
CIGAR_RESULT_DTYPE = np.dtype([("status", "<i4"), ("cost", "<i4"), ("n_ops", "<u4"), ("walk_len", "<u4"),
                               ("walk_begin", "<u4"), ("walk_end", "<u4")])
GWFA_CIGAR_INS, GWFA_CIGAR_DEL, GWFA_CIGAR_EQ, GWFA_CIGAR_DIFF = 1, 2, 7, 8
CIGAR_CHARS = {GWFA_CIGAR_INS: "I", GWFA_CIGAR_DEL: "D", GWFA_CIGAR_EQ: "=", GWFA_CIGAR_DIFF: "X"}


class gwfa_opts(ctypes.Structure):
    _fields_ = [("max_lag", ctypes.c_int32), ("traceback", ctypes.c_int32),
                ("max_score", ctypes.c_int32), ("wait_limit", ctypes.c_int32), ("ends", ctypes.c_int32),
                ("evict_lag", ctypes.c_int32), ("evict_every", ctypes.c_int32)]


# formulation variants (gwfa_opts.ends flags)
GWFA_FREE_START, GWFA_FREE_END, GWFA_EXTEND = 1, 2, 4


class gwfa_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("edit_distance", ctypes.c_int32),
                ("is_upper_bound", ctypes.c_int32), ("n_scores", ctypes.c_uint32),
                ("cells", ctypes.c_uint64), ("visited", ctypes.c_uint64),
                ("peak_frontier", ctypes.c_uint32), ("device_us", ctypes.c_uint32),
                ("pruned", ctypes.c_uint64), ("spills", ctypes.c_uint64), ("evicted", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class gwfa_graph_info(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_uint32), ("max_out_degree", ctypes.c_uint32),
                ("n_arcs", ctypes.c_uint64), ("total_bases", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64), ("device", ctypes.c_int32),
                ("has_cycles", ctypes.c_int32)]


class gwfa_tier(ctypes.Structure):
    _fields_ = [("ctas", ctypes.c_uint32), ("log2_tiles", ctypes.c_uint32),
                ("threads", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class gwfa_engine_config(ctypes.Structure):
    _fields_ = [("n_tiers", ctypes.c_uint32), ("tiers", gwfa_tier * GWFA_MAX_TIERS),
                ("wide", gwfa_tier), ("huge", gwfa_tier), ("threads", ctypes.c_uint32),
                ("prune_slabs", ctypes.c_uint32),
                ("max_queries", ctypes.c_uint64), ("max_bases", ctypes.c_uint64)]


class gwfa_schedule(ctypes.Structure):
    _fields_ = [("n_huge", ctypes.c_uint32), ("n_wide", ctypes.c_uint32)]


def _sched(n_huge: int, n_wide: int):
    return ctypes.byref(gwfa_schedule(int(n_huge), int(n_wide))) if (n_huge or n_wide) else None


# every symbol include/gwfa.h declares, with its ctypes signature
_P = ctypes.c_void_p
_u32, _u64, _i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32
SIGNATURES = {
    "gwfa_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "gwfa_graph_create": ([_u32, _P, _P, _u64, _P, _P, ctypes.c_int, ctypes.POINTER(_P)], ctypes.c_int),
    "gwfa_graph_destroy": ([_P], ctypes.c_int),
    "gwfa_graph_get_info": ([_P, ctypes.POINTER(gwfa_graph_info)], ctypes.c_int),
    "gwfa_align": ([_P, _P, _u32, _u32, _u32, ctypes.POINTER(gwfa_opts), ctypes.POINTER(gwfa_result)],
                   ctypes.c_int),
    "gwfa_engine_default_config": ([_P, ctypes.c_int, ctypes.POINTER(gwfa_engine_config)], ctypes.c_int),
    "gwfa_engine_create": ([_P, ctypes.POINTER(gwfa_engine_config), ctypes.POINTER(_P)], ctypes.c_int),
    "gwfa_engine_destroy": ([_P], ctypes.c_int),
    "gwfa_engine_device_bytes": ([_P], _u64),
    "gwfa_align_batch": ([_P, _u32, _P, _P, _P, _P, _P, _P, ctypes.POINTER(gwfa_opts), _P, _P],
                         ctypes.c_int),
    "gwfa_pack_queries_device": ([_u32, _P, _P, _P, _P, _P], ctypes.c_int),
    "gwfa_align_batch_device": ([_P, _u32, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(gwfa_opts), _P,
                                 _P], ctypes.c_int),
    "gwfa_engine_last_launches": ([_P], _u32),
    "gwfa_engine_set_stats": ([_P, _P], ctypes.c_int),
}
SIGNATURES.update({
    "gwfa_engine_last_retries": ([_P, _P], ctypes.c_int),
    "gwfa_model_create": ([_P, _u64, ctypes.POINTER(_P)], ctypes.c_int),
    "gwfa_model_destroy": ([_P], ctypes.c_int),
    "gwfa_model_set_params": ([_P, _P, _u32], ctypes.c_int),
    "gwfa_model_get_params": ([_P, _P, _u32], ctypes.c_int),
    "gwfa_model_set_normalization": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "gwfa_model_features_device": ([_P, _u32, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "gwfa_model_predict_device": ([_P, _u32, _P, _P, _P], ctypes.c_int),
    "gwfa_model_gradient_device": ([_P, _u32, _P, _P, _P, _P, _P], ctypes.c_int),
    "gwfa_model_train_device": ([_P, _u32, _P, _P, _u32, _u32, ctypes.c_float, _u64, _P, _P],
                                ctypes.c_int),
    "gwfa_plan_schedule": ([_u32, _P, _u64, _u64, _P, _P], ctypes.c_int),
    "gwfa_cigar_create": ([_P, _u32, _u64, ctypes.POINTER(_P)], ctypes.c_int),
    "gwfa_cigar_destroy": ([_P], ctypes.c_int),
    "gwfa_cigar_device": ([_P, _u32, _P, _P, _P, _P, _u32, _P, _P, _u32, _i32, _P, _P], ctypes.c_int),
})



class gwfa_server_config(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in ("threads", "ctas_small", "log2_small", "ctas_big",
                                                 "log2_big", "ring_slots", "max_query_len", "idle_us",
                                                 "big_length")]


class gwfa_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "completed", "requeued", "launches",
                                                 "in_flight", "device_bytes")]


SIGNATURES.update({
    "gwfa_model_save": ([_P, ctypes.c_char_p], ctypes.c_int),
    "gwfa_model_load": ([_P, ctypes.c_char_p], ctypes.c_int),
    "gwfa_measure_int_peak": ([ctypes.c_int, _u32, _u32, ctypes.POINTER(ctypes.c_float),
                               ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "gwfa_align_noalloc": ([_P, _u32, _P, _P, _P, _P, _P, _u32, ctypes.POINTER(gwfa_opts), _P, _P],
                           ctypes.c_int),
    "gwfa_align_path": ([_P, _P, _u32, _u32, _u32, ctypes.POINTER(gwfa_opts), ctypes.POINTER(gwfa_result),
                         _P, _u32, ctypes.POINTER(_u32)], ctypes.c_int),
    "gwfa_engine_set_paths": ([_P, _P, _u32, _P], ctypes.c_int),
    "gwfa_model_predict_host": ([_P, _P, _u32, _u32, _u32, _P], ctypes.c_int),
    "gwfa_server_default_config": ([_P, ctypes.POINTER(gwfa_server_config)], ctypes.c_int),
    "gwfa_server_create": ([_P, ctypes.POINTER(gwfa_server_config), ctypes.POINTER(gwfa_opts), _P,
                            ctypes.POINTER(_P)], ctypes.c_int),
    "gwfa_submit": ([_P, _P, _u32, _u32, _u32, ctypes.POINTER(_u64)], ctypes.c_int),
    "gwfa_poll": ([_P, _u64, ctypes.POINTER(gwfa_result)], ctypes.c_int),
    "gwfa_wait": ([_P, _u64, _u32, ctypes.POINTER(gwfa_result)], ctypes.c_int),
    "gwfa_poll_many": ([_P, _u32, _P, _P, _P, ctypes.POINTER(_u32)], ctypes.c_int),
    "gwfa_server_get_stats": ([_P, ctypes.POINTER(gwfa_server_stats)], ctypes.c_int),
    "gwfa_server_destroy": ([_P], ctypes.c_int),
})
MODEL_FEATURES, MODEL_TARGETS, MODEL_PARAMS = 6, 4, 1412
TARGET_NAMES = ("edit_distance", "peak_frontier", "visited", "cells")
STAT_FIELDS = ("extend_ns", "expand_ns", "rounds", "extend_tiles", "expand_tiles", "max_tiles",
               "hash_tiles", "scores")

_lib = None


class GwfaError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status})" if what else strerror(status))


def load(path: str | None = None):
    """Load libgwfa.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with paper_2206_13574_gb300._build.build()")
    lib = ctypes.CDLL(p)
    for name, (args, res) in SIGNATURES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def strerror(status: int) -> str:
    if _lib is None:
        return f"status {status}"
    return _lib.gwfa_strerror(status).decode()


def _check(st: int, what: str):
    if st != GWFA_OK:
        raise GwfaError(st, what)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _opts(max_lag: int, max_score: int, traceback: int = 0, ends: int = 0, evict_lag: int = 0,
          evict_every: int = 0) -> gwfa_opts:
    return gwfa_opts(int(max_lag), int(traceback), int(max_score), 0, int(ends), int(evict_lag), int(evict_every))


class Graph:
    """A sequence graph resident on one GPU (gwfa_graph_create)."""

    def __init__(self, seq, off, arc_src, arc_dst, device: int = 0):
        lib = load()
        self._seq = _c(seq, np.uint8)
        self._off = _c(off, np.uint64)
        src = _c(arc_src, np.uint32)
        dst = _c(arc_dst, np.uint32)
        h = _P()
        _check(lib.gwfa_graph_create(len(self._off) - 1, self._seq.ctypes.data, self._off.ctypes.data,
                                     len(src), src.ctypes.data, dst.ctypes.data, device,
                                     ctypes.byref(h)), "gwfa_graph_create")
        self.handle = h
        self.device = device

    @classmethod
    def from_synth(cls, g, device: int = 0) -> "Graph":
        return cls(g.seq, g.off, g.arc_src, g.arc_dst, device)

    def info(self) -> dict:
        i = gwfa_graph_info()
        _check(load().gwfa_graph_get_info(self.handle, ctypes.byref(i)), "gwfa_graph_get_info")
        return {k: int(getattr(i, k)) for k, _ in i._fields_}

    def align(self, q: bytes, v_s: int, v_e: int, max_lag: int = 0, max_score: int = -1,
              ends: int = 0, evict_lag: int = 0, evict_every: int = 0) -> dict:
        """Plain path (gwfa_align): one query, one kernel launch, synchronous."""
        r = gwfa_result()
        o = _opts(max_lag, max_score, 0, ends, evict_lag, evict_every)
        qb = bytes(q)
        _check(load().gwfa_align(self.handle, qb, len(qb), v_s, v_e, ctypes.byref(o), ctypes.byref(r)),
               "gwfa_align")
        return r.as_dict()

    def align_path(self, q: bytes, v_s: int, v_e: int, max_score: int = -1, path_cap: int = 1 << 16,
                   ends: int = 0, max_lag: int = 0):
        """(result, walk) with the optimal walk's vertex ids (gwfa_align_path); with
        max_lag > 0 the walk the lag-pruned wavefront reached the end along."""
        r = gwfa_result()
        o = _opts(max_lag, max_score, 0, ends)
        qb = bytes(q)
        path = np.zeros(path_cap, dtype=np.uint32)
        plen = _u32()
        _check(load().gwfa_align_path(self.handle, qb, len(qb), v_s, v_e, ctypes.byref(o), ctypes.byref(r),
                                      path.ctypes.data, path_cap, ctypes.byref(plen)), "gwfa_align_path")
        return r.as_dict(), path[:min(plen.value, path_cap)].copy()

    def close(self):
        if getattr(self, "handle", None):
            load().gwfa_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def default_config(graph: Graph, prune: bool = False) -> gwfa_engine_config:
    c = gwfa_engine_config()
    _check(load().gwfa_engine_default_config(graph.handle, int(prune), ctypes.byref(c)),
           "gwfa_engine_default_config")
    return c


class Engine:
    """Batched alignment workspace (gwfa_engine_create)."""

    def __init__(self, graph: Graph, prune: bool = False, config: gwfa_engine_config | None = None):
        lib = load()
        self.graph = graph
        self.config = config if config is not None else default_config(graph, prune)
        h = _P()
        _check(lib.gwfa_engine_create(graph.handle, ctypes.byref(self.config), ctypes.byref(h)),
               "gwfa_engine_create")
        self.handle = h

    @property
    def device_bytes(self) -> int:
        return int(load().gwfa_engine_device_bytes(self.handle))

    @property
    def last_launches(self) -> int:
        return int(load().gwfa_engine_last_launches(self.handle))

    def last_retries(self) -> np.ndarray:
        """Queries each tier handed to the next in the last batch call (synchronises)."""
        out = np.zeros(GWFA_MAX_TIERS, dtype=np.uint32)
        _check(load().gwfa_engine_last_retries(self.handle, out.ctypes.data), "gwfa_engine_last_retries")
        return out

    def set_paths(self, d_paths: int | None, path_cap: int = 0, d_path_len: int | None = None):
        """Walk output for batches with traceback (device buffers, or None to stop)."""
        _check(load().gwfa_engine_set_paths(self.handle, d_paths or None, path_cap, d_path_len or None),
               "gwfa_engine_set_paths")

    def set_stats(self, d_stats: int | None):
        """Per-query statistics into device memory (8 uint64 per query id), or None to stop."""
        _check(load().gwfa_engine_set_stats(self.handle, d_stats or None), "gwfa_engine_set_stats")

    def align_batch(self, seq, off, v_s, v_e, order=None, max_lag: int = 0, max_score: int = -1,
                    stream: int = 0, out: np.ndarray | None = None, n_wide: int = 0,
                    n_huge: int = 0, ends: int = 0, evict_lag: int = 0, evict_every: int = 0) -> np.ndarray:
        """Host buffers in, host results out (gwfa_align_batch)."""
        seq = _c(seq, np.uint8)
        off = _c(off, np.uint64)
        vs = _c(v_s, np.uint32)
        ve = _c(v_e, np.uint32)
        n = len(vs)
        res = out if out is not None else np.zeros(n, dtype=RESULT_DTYPE)
        o = _opts(max_lag, max_score, 0, ends, evict_lag, evict_every)
        od = None if order is None else _c(order, np.uint32)
        _check(load().gwfa_align_batch(self.handle, n, seq.ctypes.data, off.ctypes.data, vs.ctypes.data,
                                       ve.ctypes.data, None if od is None else od.ctypes.data,
                                       _sched(n_huge, n_wide),
                                       ctypes.byref(o), res.ctypes.data, stream or None),
               "gwfa_align_batch")
        return res

    def align_batch_device(self, n: int, d_words: int, d_q_off: int, d_v_s: int, d_v_e: int,
                           d_order: int | None, d_status: int | None, d_out: int,
                           max_lag: int = 0, max_score: int = -1, stream: int = 0, n_wide: int = 0,
                           traceback: bool = False, n_huge: int = 0, ends: int = 0, evict_lag: int = 0,
                           evict_every: int = 0):
        """Device pointers in and out, asynchronous on `stream` (gwfa_align_batch_device)."""
        o = _opts(max_lag, max_score, int(traceback), ends, evict_lag, evict_every)
        _check(load().gwfa_align_batch_device(self.handle, n, d_words, d_q_off, d_v_s, d_v_e,
                                              d_order or None, _sched(n_huge, n_wide), d_status or None,
                                              ctypes.byref(o),
                                              d_out, stream or None),
               "gwfa_align_batch_device")

    def close(self):
        if getattr(self, "handle", None):
            load().gwfa_engine_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pack_queries_device(n: int, d_q: int, d_q_off: int, d_words: int, d_status: int | None,
                        stream: int = 0):
    _check(load().gwfa_pack_queries_device(n, d_q, d_q_off, d_words, d_status or None, stream or None),
           "gwfa_pack_queries_device")


def words_needed(n_queries: int, n_bases: int) -> int:
    """Words of the packed query buffer (query i starts at word (q_off[i] >> 4) + i)."""
    return (n_bases >> 4) + n_queries + 2


class DeviceBatch:
    """A query batch resident in HBM as torch tensors: ASCII, offsets, packed words, ids."""

    def __init__(self, queries, device: int = 0, order=None, stream=None):
        import torch
        dev = torch.device("cuda", device)
        self.n = len(queries.v_s)
        self.n_bases = int(queries.off[-1])
        self.q = torch.from_numpy(_c(queries.seq, np.uint8)).to(dev)
        self.q_off = torch.from_numpy(_c(queries.off, np.uint64).view(np.int64)).to(dev)
        self.v_s = torch.from_numpy(_c(queries.v_s, np.uint32).view(np.int32)).to(dev)
        self.v_e = torch.from_numpy(_c(queries.v_e, np.uint32).view(np.int32)).to(dev)
        self.order = None if order is None else torch.from_numpy(
            _c(order, np.uint32).view(np.int32)).to(dev)
        self.words = torch.empty(words_needed(self.n, self.n_bases), dtype=torch.int32, device=dev)
        self.status = torch.empty(self.n, dtype=torch.int32, device=dev)
        self.out = torch.empty(self.n * RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        pack_queries_device(self.n, self.q.data_ptr(), self.q_off.data_ptr(), self.words.data_ptr(),
                            self.status.data_ptr(), st.cuda_stream)

    def run(self, engine: Engine, max_lag: int = 0, max_score: int = -1, stream=None, n_wide: int = 0,
            traceback: bool = False, n_huge: int = 0, ends: int = 0, evict_lag: int = 0,
            evict_every: int = 0):
        import torch
        st = stream if stream is not None else torch.cuda.current_stream(self.q.device)
        engine.align_batch_device(self.n, self.words.data_ptr(), self.q_off.data_ptr(),
                                  self.v_s.data_ptr(), self.v_e.data_ptr(),
                                  None if self.order is None else self.order.data_ptr(),
                                  self.status.data_ptr(), self.out.data_ptr(), max_lag, max_score,
                                  st.cuda_stream, n_wide, traceback, n_huge, ends, evict_lag, evict_every)

    def results(self) -> np.ndarray:
        return self.out.cpu().numpy().view(RESULT_DTYPE)


class CostModel:
    """The learned cost model (gwfa_model_*): features, predictions and training on
    the device; parameters are fp32 numpy arrays on the host side."""

    def __init__(self, graph: Graph, seed: int = 1):
        h = _P()
        _check(load().gwfa_model_create(graph.handle, seed, ctypes.byref(h)), "gwfa_model_create")
        self.handle = h
        self.graph = graph
        self.norm = None

    def features(self, batch: "DeviceBatch", stream=None):
        import torch
        f = torch.empty((batch.n, MODEL_FEATURES), dtype=torch.float32, device=batch.q.device)
        st = stream if stream is not None else torch.cuda.current_stream(batch.q.device)
        _check(load().gwfa_model_features_device(self.handle, batch.n, batch.words.data_ptr(),
                                                 batch.q_off.data_ptr(), batch.v_s.data_ptr(),
                                                 batch.v_e.data_ptr(), f.data_ptr(), st.cuda_stream),
               "gwfa_model_features_device")
        return f

    def set_normalization(self, fmean, fstd, tmean, tstd):
        arrs = [_c(a, np.float32) for a in (fmean, fstd, tmean, tstd)]
        _check(load().gwfa_model_set_normalization(self.handle, *[a.ctypes.data for a in arrs]),
               "gwfa_model_set_normalization")
        self.norm = arrs

    def predict(self, feat, stream=None):
        import torch
        p = torch.empty((feat.shape[0], MODEL_TARGETS), dtype=torch.float32, device=feat.device)
        st = stream if stream is not None else torch.cuda.current_stream(feat.device)
        _check(load().gwfa_model_predict_device(self.handle, feat.shape[0], feat.data_ptr(), p.data_ptr(),
                                                st.cuda_stream), "gwfa_model_predict_device")
        return p

    def gradient(self, feat, target):
        import torch
        g = np.zeros(MODEL_PARAMS, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        st = torch.cuda.current_stream(feat.device).cuda_stream
        _check(load().gwfa_model_gradient_device(self.handle, feat.shape[0], feat.data_ptr(),
                                                 target.data_ptr(), g.ctypes.data, loss.ctypes.data,
                                                 st or None), "gwfa_model_gradient_device")
        return g, float(loss[0])

    def train(self, feat, target, steps: int, batch: int = 512, lr: float = 3e-3, seed: int = 7):
        import torch
        losses = np.zeros(steps, dtype=np.float32)
        st = torch.cuda.current_stream(feat.device).cuda_stream
        _check(load().gwfa_model_train_device(self.handle, feat.shape[0], feat.data_ptr(), target.data_ptr(),
                                              steps, batch, lr, seed, losses.ctypes.data, st or None),
               "gwfa_model_train_device")
        return losses

    def predict_host(self, q: bytes, v_s: int, v_e: int) -> np.ndarray:
        """The four predictions for one ASCII query, evaluated on the host in fp32
        (gwfa_model_predict_host: the server's admission path)."""
        out = np.zeros(MODEL_TARGETS, dtype=np.float32)
        qb = bytes(q)
        _check(load().gwfa_model_predict_host(self.handle, qb, len(qb), v_s, v_e, out.ctypes.data),
               "gwfa_model_predict_host")
        return out

    def save(self, path: str):
        """Weights and normalisation to a file (gwfa_model_save)."""
        _check(load().gwfa_model_save(self.handle, os.fsencode(path)), "gwfa_model_save")

    def load(self, path: str):
        """Weights and normalisation from a file written by save (gwfa_model_load)."""
        _check(load().gwfa_model_load(self.handle, os.fsencode(path)), "gwfa_model_load")
        # the file's normalisation block follows the tag, three counts and the weights
        raw = np.fromfile(path, dtype=np.float32, offset=8 + 12 + 4 * MODEL_PARAMS)
        nf, nt = MODEL_FEATURES, MODEL_TARGETS
        cuts = np.cumsum([nf, nf, nt, nt])
        self.norm = [raw[0:cuts[0]].copy(), raw[cuts[0]:cuts[1]].copy(), raw[cuts[1]:cuts[2]].copy(),
                     raw[cuts[2]:cuts[3]].copy()]

    @property
    def params(self) -> np.ndarray:
        w = np.zeros(MODEL_PARAMS, dtype=np.float32)
        _check(load().gwfa_model_get_params(self.handle, w.ctypes.data, MODEL_PARAMS), "gwfa_model_get_params")
        return w

    @params.setter
    def params(self, w):
        w = _c(w, np.float32)
        _check(load().gwfa_model_set_params(self.handle, w.ctypes.data, len(w)), "gwfa_model_set_params")

    def close(self):
        if getattr(self, "handle", None):
            load().gwfa_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_schedule(pred: np.ndarray, tier0_tiles: int, wide_tiles: int = 0):
    """(order, n_huge, n_wide) from predictions (n x 4, log1p units): gwfa_plan_schedule."""
    pred = _c(pred, np.float32)
    n = pred.shape[0]
    order = np.zeros(n, dtype=np.uint32)
    sc = gwfa_schedule()
    _check(load().gwfa_plan_schedule(n, pred.ctypes.data, int(tier0_tiles), int(wide_tiles),
                                     order.ctypes.data, ctypes.byref(sc)), "gwfa_plan_schedule")
    return order, int(sc.n_huge), int(sc.n_wide)


class Cigar:
    """Base-level alignment of queries to their walks (gwfa_cigar_*): a workspace of
    `ctas` x `workspace_bytes` on the graph's GPU (0 = library defaults)."""

    def __init__(self, graph: Graph, ctas: int = 0, workspace_bytes: int = 0):
        h = _P()
        _check(load().gwfa_cigar_create(graph.handle, int(ctas), int(workspace_bytes), ctypes.byref(h)),
               "gwfa_cigar_create")
        self.graph = graph
        self.handle = h

    def run_device(self, n: int, d_words: int, d_q_off: int, d_res: int, d_paths: int, path_cap: int,
                   d_path_len: int, d_cigar: int | None, cigar_cap: int, d_out: int, stream: int = 0,
                   ends: int = 0):
        _check(load().gwfa_cigar_device(self.handle, n, d_words, d_q_off, d_res, d_paths, path_cap,
                                        d_path_len, d_cigar or None, cigar_cap, int(ends), d_out, stream or None),
               "gwfa_cigar_device")

    def run(self, batch: "DeviceBatch", paths, path_len, path_cap: int, cigar_cap: int = 1024,
            stream=None, ends: int = 0):
        """CIGARs of a batch after a traceback run whose walks are in the device
        tensors `paths` / `path_len`; returns (ops tensor n x cigar_cap, results tensor)."""
        import torch
        dev = batch.q.device
        ops = torch.zeros(batch.n * cigar_cap, dtype=torch.int32, device=dev)
        out = torch.empty(batch.n * CIGAR_RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        self.run_device(batch.n, batch.words.data_ptr(), batch.q_off.data_ptr(), batch.out.data_ptr(),
                        paths.data_ptr(), path_cap, path_len.data_ptr(), ops.data_ptr(), cigar_cap,
                        out.data_ptr(), st.cuda_stream, ends)
        return ops, out

    def close(self):
        if getattr(self, "handle", None):
            load().gwfa_cigar_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cigar_string(ops) -> str:
    """Text form of CIGAR operations (uint32 length << 4 | op)."""
    return "".join(f"{int(o) >> 4}{CIGAR_CHARS[int(o) & 15]}" for o in np.asarray(ops, dtype=np.uint32))


class Server:
    """Continuous-batching server over a resident graph (gwfa_server_*)."""

    def __init__(self, graph: Graph, config: gwfa_server_config | None = None, max_lag: int = 0,
                 max_score: int = -1, model: "CostModel | None" = None):
        lib = load()
        if config is None:
            config = gwfa_server_config()
            _check(lib.gwfa_server_default_config(graph.handle, ctypes.byref(config)),
                   "gwfa_server_default_config")
        self.config = config
        self.graph = graph
        self.model = model
        o = _opts(max_lag, max_score)
        h = _P()
        _check(lib.gwfa_server_create(graph.handle, ctypes.byref(config), ctypes.byref(o),
                                      model.handle if model is not None else None, ctypes.byref(h)),
               "gwfa_server_create")
        self.handle = h

    def submit(self, q: bytes, v_s: int, v_e: int) -> int | None:
        """Ticket, or None when the ring is full (retry later)."""
        t = ctypes.c_uint64()
        st = load().gwfa_submit(self.handle, q, len(q), v_s, v_e, ctypes.byref(t))
        if st == GWFA_PENDING:
            return None
        _check(st, "gwfa_submit")
        return int(t.value)

    def poll(self, ticket: int) -> dict | None:
        r = gwfa_result()
        st = load().gwfa_poll(self.handle, ticket, ctypes.byref(r))
        if st == GWFA_PENDING:
            return None
        _check(st, "gwfa_poll")
        return r.as_dict()

    def poll_many(self, tickets: np.ndarray, out: np.ndarray, done: np.ndarray) -> int:
        """Poll every ticket not yet done; results into out (RESULT_DTYPE), flags into done."""
        k = _u32()
        _check(load().gwfa_poll_many(self.handle, len(tickets), tickets.ctypes.data, out.ctypes.data,
                                     done.ctypes.data, ctypes.byref(k)), "gwfa_poll_many")
        return int(k.value)

    def wait(self, ticket: int, timeout_ms: int = 60000) -> dict:
        r = gwfa_result()
        _check(load().gwfa_wait(self.handle, ticket, timeout_ms, ctypes.byref(r)), "gwfa_wait")
        return r.as_dict()

    def stats(self) -> dict:
        s = gwfa_server_stats()
        _check(load().gwfa_server_get_stats(self.handle, ctypes.byref(s)), "gwfa_server_get_stats")
        return {k: int(getattr(s, k)) for k, _ in s._fields_}

    def close(self):
        if getattr(self, "handle", None):
            load().gwfa_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def align_noalloc(graph: Graph, batch: "DeviceBatch", log2_tiles: int = 0, max_lag: int = 0,
                  max_score: int = -1, stream=None) -> int:
    """gwfa_align_noalloc on a DeviceBatch, results into batch.out; returns the status.

    For callers that cannot let the library allocate device memory: the scratch is a
    fixed 32 MiB array inside the library, shared by all calls (serialise them)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream(batch.q.device)
    o = _opts(max_lag, max_score)
    return int(load().gwfa_align_noalloc(graph.handle, batch.n, batch.words.data_ptr(), batch.q_off.data_ptr(),
                                         batch.v_s.data_ptr(), batch.v_e.data_ptr(), batch.status.data_ptr(),
                                         log2_tiles,
                                         ctypes.byref(o), batch.out.data_ptr(), st.cuda_stream or None))


def measure_int_peak(device: int = 0, iters: int = 20000, blocks_per_sm: int = 2) -> dict:
    """ALU-pipe ceiling of the GPU from the library's lop3 microbenchmark
    (gwfa_measure_int_peak): warp instructions per second, and per SM per cycle at
    the SM clock the caller reports."""
    ms = ctypes.c_float()
    n = ctypes.c_uint64()
    _check(load().gwfa_measure_int_peak(device, blocks_per_sm, iters, ctypes.byref(ms), ctypes.byref(n)),
           "gwfa_measure_int_peak")
    return {"warp_insts": int(n.value), "ms": float(ms.value),
            "warp_inst_per_s": int(n.value) / (float(ms.value) * 1e-3)}
