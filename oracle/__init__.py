"""CPU oracle for the graph wavefront alignment library -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the benchmark's CPU-baseline /
reference leg may import this package.  The library itself never does: it has
no CPU fallback.

The arithmetic lives in `gwfa_oracle.c` (plain C, built by `build()` with gcc);
this module only marshals arguments.  `brute.py` holds the pure-python
brute-force pins used on tiny graphs.

Pins (what ties each function to something other than itself; see tests/):
  * oracle_dp      - brute-force walk enumeration on tiny DAGs and cyclic graphs;
                     Levenshtein on single-vertex and chain graphs (Sec. 2.2:
                     a chain of vertices is one string); d = 0 for error-free
                     walk copies; |q| = 0 gives the shortest spelled walk.
  * oracle_gwfa    - exact mode equals oracle_dp (Gwfa is exact, Sec. 2.4);
                     hand-traced work counts (tests/golden/); pruned mode is an
                     upper bound (Sec. 2.5) and equals exact mode when a_diff
                     exceeds every a.  The tie rules for W~ in pruned mode are
                     a reading of the paper; their order independence is pinned
                     by arc-order permutations, against a planted first-spill-
                     wins rule (GWFA_ORACLE_PLANT_FIRST_TIE, tests only).
  * levenshtein    - textbook values and a python restatement.
  * memory bound   - (evict_lag) removes H~ entries behind the lag: pinned by the
                     upper-bound property (never below the exact distance), by
                     equality with the unbounded run when evict_lag exceeds every
                     a, and by fewer entries kept at the end.
  * ends variants  - (free walk start / free walk end / no end vertex, Sec. 2.1)
                     the DP against brute-force enumeration of walks and of
                     their skipped prefixes / suffixes (brute.py); the variant
                     Gwfa against the variant DP; closed forms: free start and
                     end on one vertex is the best substring match, a query
                     spelled inside a vertex gives 0.
"""
from __future__ import annotations

FREE_START, FREE_END, EXTEND = 1, 2, 4   # formulation variants (flags)

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gwfa_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: it also builds on the Arm GPU host)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class Stats(ctypes.Structure):
    _fields_ = [("distance", ctypes.c_int64), ("is_upper_bound", ctypes.c_int64),
                ("n_scores", ctypes.c_int64), ("cells", ctypes.c_int64),
                ("peak", ctypes.c_int64), ("visited", ctypes.c_int64),
                ("pruned", ctypes.c_int64), ("spills", ctypes.c_int64), ("evicted", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            u32, u64, i64 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64
            lib.oracle_levenshtein.argtypes = [P, u64, P, u64]
            lib.oracle_levenshtein.restype = i64
            lib.oracle_dp.argtypes = [u32, P, P, u64, P, P, P, u64, u32, u32]
            lib.oracle_dp.restype = i64
            lib.oracle_gwfa.argtypes = [u32, P, P, u64, P, P, P, u64, u32, u32, i64, i64,
                                        ctypes.POINTER(Stats)]
            lib.oracle_gwfa.restype = ctypes.c_int
            lib.oracle_dp_ends.argtypes = [u32, P, P, u64, P, P, P, u64, u32, u32, ctypes.c_int]
            lib.oracle_dp_ends.restype = i64
            lib.oracle_gwfa_ends.argtypes = [u32, P, P, u64, P, P, P, u64, u32, u32, i64, i64, ctypes.c_int,
                                             ctypes.POINTER(Stats)]
            lib.oracle_gwfa_ends.restype = ctypes.c_int
            lib.oracle_gwfa_ex.argtypes = [u32, P, P, u64, P, P, P, u64, u32, u32, i64, i64, ctypes.c_int,
                                           i64, i64, ctypes.POINTER(Stats)]
            lib.oracle_gwfa_ex.restype = ctypes.c_int
            lib.oracle_stats_size.restype = u64
            assert lib.oracle_stats_size() == ctypes.sizeof(Stats)
            _lib = lib
    return _lib


def _buf(x: bytes | np.ndarray):
    if isinstance(x, (bytes, bytearray)):
        a = np.frombuffer(bytes(x), dtype=np.uint8)
    else:
        a = np.ascontiguousarray(x)
    return a, a.ctypes.data


class GraphArgs:
    """Keeps the contiguous arrays of a graph alive for repeated oracle calls."""

    def __init__(self, g):
        self.seq = np.ascontiguousarray(g.seq, dtype=np.uint8)
        self.off = np.ascontiguousarray(g.off, dtype=np.uint64)
        self.src = np.ascontiguousarray(g.arc_src, dtype=np.uint32)
        self.dst = np.ascontiguousarray(g.arc_dst, dtype=np.uint32)
        self.nv = len(self.off) - 1
        self.na = len(self.src)

    def args(self):
        return (self.nv, self.seq.ctypes.data, self.off.ctypes.data, self.na,
                self.src.ctypes.data, self.dst.ctypes.data)


def _gargs(g):
    return g if isinstance(g, GraphArgs) else GraphArgs(g)


def levenshtein(x: bytes, y: bytes) -> int:
    lib = _load()
    ax, px = _buf(x)
    ay, py = _buf(y)
    return int(lib.oracle_levenshtein(px, len(ax), py, len(ay)))


def dp_distance(g, q: bytes, v_s: int, v_e: int, ends: int = 0) -> int:
    """Eq. 1 distance (negative = error status); `ends` = variant flags."""
    lib = _load()
    ga = _gargs(g)
    aq, pq = _buf(q)
    if ends:
        return int(lib.oracle_dp_ends(*ga.args(), pq, len(aq), v_s, v_e, ends))
    return int(lib.oracle_dp(*ga.args(), pq, len(aq), v_s, v_e))


def gwfa(g, q: bytes, v_s: int, v_e: int, a_diff: int = 0, max_score: int = -1, ends: int = 0,
         evict_lag: int = 0, evict_every: int = 0) -> dict:
    """Alg. 1-4 on the CPU; returns the distance (or status) and the work counts.
    evict_lag > 0 (with a_diff > 0) bounds H~: every evict_every scores the entries
    outside Q lagging a_max by evict_lag or more are removed."""
    lib = _load()
    ga = _gargs(g)
    aq, pq = _buf(q)
    st = Stats()
    if evict_lag:
        lib.oracle_gwfa_ex(*ga.args(), pq, len(aq), v_s, v_e, a_diff, max_score, ends, evict_lag, evict_every,
                           ctypes.byref(st))
    elif ends:
        lib.oracle_gwfa_ends(*ga.args(), pq, len(aq), v_s, v_e, a_diff, max_score, ends, ctypes.byref(st))
    else:
        lib.oracle_gwfa(*ga.args(), pq, len(aq), v_s, v_e, a_diff, max_score, ctypes.byref(st))
    return st.as_dict()


def gwfa_many(g, queries, idx, a_diff: int = 0, threads: int | None = None, ends: int = 0,
              evict_lag: int = 0, evict_every: int = 0) -> list[dict]:
    """oracle gwfa over queries[idx] with a thread pool (ctypes releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    ga = _gargs(g)
    threads = threads or os.cpu_count() or 1
    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(lambda i: gwfa(ga, queries.query(int(i)), int(queries.v_s[i]),
                                          int(queries.v_e[i]), a_diff, ends=ends, evict_lag=evict_lag,
                                          evict_every=evict_every), idx))


def dp_many(g, queries, idx, threads: int | None = None) -> list[int]:
    from concurrent.futures import ThreadPoolExecutor
    ga = _gargs(g)
    threads = threads or os.cpu_count() or 1
    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(lambda i: dp_distance(ga, queries.query(int(i)), int(queries.v_s[i]),
                                                 int(queries.v_e[i])), idx))
