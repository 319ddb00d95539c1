"""Seeded synthetic sequence graphs and queries.

This module only draws inputs: it holds none of the alignment arithmetic, so the
CUDA path and the CPU oracle can both be fed from it without sharing any of the
method's code.

Randomness comes from one counter-based generator written here from its
published definition (SplitMix64, Steele, Lea & Flood, OOPSLA 2014): output t of
a stream with key K is mix(K + t * 0x9E3779B97F4A7C15).  Every stream is
identified by (seed, stream id), so the bytes are identical on every machine and
every numpy version.

Graph model (a chain of "sites" along a random backbone, vertex ids in backbone
order so that ids are a topological order apart from loop back-arcs):

* segment  - one backbone slice between two sites;
* snp      - two 1-bp vertices (backbone base / a different base) in parallel;
* indel    - one skippable vertex: half the time new random bases (an
             insertion), half the time backbone bases (a deletion);
* alt      - a backbone branch of U[a,b] bp in parallel with an independent
             random branch of U[a,b] bp;
* loop     - a tandem-repeat unit vertex (backbone bases) with a self arc; a
             walk takes it 1..10 times.

Queries are the spelled sequence of a contiguous sub-walk that starts at a
segment vertex and ends at the first vertex at which the spelled length reaches
the target, with single-base errors injected afterwards.  v_s / v_e are the first
and last vertex of that sub-walk, so an error-free query aligns at distance 0
(Def. 2 penalises unaligned ends).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_ACGT = np.frombuffer(b"ACGT", dtype=np.uint8)
_MASK = 0xFFFFFFFFFFFFFFFF


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Rng:
    """SplitMix64 stream; draws are vectorised and independent of numpy's RNGs."""

    def __init__(self, seed: int, stream: int = 0):
        key = np.array([(seed * 0x100000001B3 + stream * 0x9E3779B1 + 1) & 0xFFFFFFFFFFFFFFFF],
                       dtype=np.uint64)
        self._key = _mix(key)[0]
        self._ctr = 0

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(self._ctr + 1, self._ctr + n + 1, dtype=np.uint64)
        self._ctr += n
        return _mix(self._key + idx * _GOLDEN)

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1)."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """n integers uniform in [lo, hi] (both ends included)."""
        span = hi - lo + 1
        return lo + np.minimum((self.uniform(n) * span).astype(np.int64), span - 1)

    def _one_u64(self) -> int:
        # the same stream as u64(1), in plain integers (scalar draws are hot in the walkers)
        self._ctr += 1
        z = (int(self._key) + self._ctr * 0x9E3779B97F4A7C15) & _MASK
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def one(self) -> float:
        return (self._one_u64() >> 11) * (1.0 / 9007199254740992.0)

    def one_int(self, lo: int, hi: int) -> int:
        span = hi - lo + 1
        return lo + min(int(self.one() * span), span - 1)

    def codes(self, n: int) -> np.ndarray:
        """n random base codes 0..3."""
        return (self.u64(n) >> np.uint64(62)).astype(np.uint8)

    def normal(self, n: int) -> np.ndarray:
        """Box-Muller standard normals."""
        u1 = np.maximum(self.uniform(n), 1e-300)
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ----------------------------------------------------------------------------
# containers


@dataclasses.dataclass
class Graph:
    """A sequence graph G(V, E, sigma): vertex labels concatenated as ASCII ACGT."""

    seq: np.ndarray        # uint8 ASCII, all labels concatenated
    off: np.ndarray        # uint64[V+1], label v is seq[off[v]:off[v+1]]
    arc_src: np.ndarray    # uint32[E]
    arc_dst: np.ndarray    # uint32[E]
    source: int = 0
    sink: int = 0
    # per-site allele structure, used only to draw walks for queries
    sites: list = dataclasses.field(default_factory=list, repr=False)

    @property
    def n_vertices(self) -> int:
        return len(self.off) - 1

    @property
    def n_arcs(self) -> int:
        return len(self.arc_src)

    def label(self, v: int) -> bytes:
        return self.seq[int(self.off[v]):int(self.off[v + 1])].tobytes()

    def lengths(self) -> np.ndarray:
        return np.diff(self.off).astype(np.int64)

    @staticmethod
    def from_lists(labels, arcs) -> "Graph":
        """Build from python lists: labels (str/bytes per vertex), arcs [(u, v)]."""
        bl = [x.encode() if isinstance(x, str) else bytes(x) for x in labels]
        off = np.zeros(len(bl) + 1, dtype=np.uint64)
        off[1:] = np.cumsum([len(x) for x in bl])
        seq = np.frombuffer(b"".join(bl), dtype=np.uint8).copy()
        src = np.array([a for a, _ in arcs], dtype=np.uint32)
        dst = np.array([b for _, b in arcs], dtype=np.uint32)
        return Graph(seq=seq, off=off, arc_src=src, arc_dst=dst, source=0,
                     sink=max(len(bl) - 1, 0))


@dataclasses.dataclass
class Queries:
    seq: np.ndarray        # uint8 ASCII, all queries concatenated
    off: np.ndarray        # uint64[Q+1]
    v_s: np.ndarray        # uint32[Q]
    v_e: np.ndarray        # uint32[Q]
    edits: np.ndarray      # int64[Q], number of single-base errors injected
    divergence: np.ndarray  # float64[Q], per-base error rate drawn for the query

    def __len__(self) -> int:
        return len(self.v_s)

    def query(self, i: int) -> bytes:
        return self.seq[int(self.off[i]):int(self.off[i + 1])].tobytes()

    def lengths(self) -> np.ndarray:
        return np.diff(self.off).astype(np.int64)

    def subset(self, idx) -> "Queries":
        idx = np.asarray(idx, dtype=np.int64)
        parts = [self.seq[int(self.off[i]):int(self.off[i + 1])] for i in idx]
        off = np.zeros(len(idx) + 1, dtype=np.uint64)
        off[1:] = np.cumsum([len(p) for p in parts]) if len(parts) else []
        seq = np.concatenate(parts) if parts else np.zeros(0, dtype=np.uint8)
        return Queries(seq=seq, off=off, v_s=self.v_s[idx].copy(), v_e=self.v_e[idx].copy(),
                       edits=self.edits[idx].copy(), divergence=self.divergence[idx].copy())


# ----------------------------------------------------------------------------
# graph generator


@dataclasses.dataclass
class GraphSpec:
    backbone: int
    gap: tuple            # (lo, hi) backbone bp between sites
    p_snp: float
    p_indel: float
    indel_len: tuple
    p_alt: float = 0.0
    alt_len: tuple = (200, 2000)
    loop_every: tuple | None = None   # (lo, hi) bp between tandem-repeat loops
    loop_unit: tuple = (2, 200)


def make_graph(spec: GraphSpec, seed: int) -> Graph:
    rng = Rng(seed, 0)
    bb = rng.codes(spec.backbone)
    labels: list[np.ndarray] = []
    arcs: list[tuple[int, int]] = []
    sites: list[tuple] = []   # ("seg", v) | ("alts", [v...], skippable) | ("loop", v)

    def add_vertex(codes: np.ndarray) -> int:
        labels.append(codes)
        return len(labels) - 1

    prev_exits: list[int] = []
    pending_skip: list[int] = []   # exits that bypass a skippable site

    def connect(entries: list[int]):
        nonlocal prev_exits, pending_skip
        for u in prev_exits + pending_skip:
            for v in entries:
                arcs.append((u, v))
        pending_skip = []

    pos = 0
    next_loop = (rng.one_int(*spec.loop_every) if spec.loop_every else None)
    srng = Rng(seed, 1)
    while pos < spec.backbone:
        gap = srng.one_int(*spec.gap)
        seg_end = min(pos + gap, spec.backbone)
        v = add_vertex(bb[pos:seg_end])
        connect([v])
        prev_exits = [v]
        sites.append(("seg", v))
        pos = seg_end
        if pos >= spec.backbone:
            break
        if next_loop is not None and pos >= next_loop:
            unit = srng.one_int(*spec.loop_unit)
            unit = min(unit, spec.backbone - pos)
            u = add_vertex(bb[pos:pos + unit])
            connect([u])
            arcs.append((u, u))
            prev_exits = [u]
            sites.append(("loop", u))
            pos += unit
            next_loop = pos + srng.one_int(*spec.loop_every)
            continue
        r = srng.one()
        if r < spec.p_snp:
            ref = int(bb[pos])
            alt = (ref + 1 + srng.one_int(0, 2)) & 3
            a = add_vertex(bb[pos:pos + 1])
            b = add_vertex(np.array([alt], dtype=np.uint8))
            connect([a, b])
            prev_exits = [a, b]
            sites.append(("alts", [a, b], False))
            pos += 1
        elif r < spec.p_snp + spec.p_indel:
            ln = srng.one_int(*spec.indel_len)
            if srng.one() < 0.5:          # insertion: new bases, backbone unchanged
                x = add_vertex(srng.codes(ln))
            else:                          # deletion: skippable backbone slice
                ln = min(ln, spec.backbone - pos)
                x = add_vertex(bb[pos:pos + ln])
                pos += ln
            skip = list(prev_exits)
            connect([x])
            prev_exits = [x]
            pending_skip = skip
            sites.append(("alts", [x], True))
        else:
            lr = min(srng.one_int(*spec.alt_len), spec.backbone - pos)
            la = srng.one_int(*spec.alt_len)
            a = add_vertex(bb[pos:pos + lr])
            b = add_vertex(srng.codes(la))
            connect([a, b])
            prev_exits = [a, b]
            sites.append(("alts", [a, b], False))
            pos += lr
    # close: a final segment so that every walk has a common sink
    tail = add_vertex(srng.codes(max(1, spec.gap[0])))
    connect([tail])
    sites.append(("seg", tail))

    lens = np.array([len(x) for x in labels], dtype=np.uint64)
    off = np.zeros(len(labels) + 1, dtype=np.uint64)
    off[1:] = np.cumsum(lens)
    seq = _ACGT[np.concatenate(labels)]
    arr = np.array(arcs, dtype=np.uint32).reshape(-1, 2)
    return Graph(seq=seq, off=off, arc_src=arr[:, 0].copy(), arc_dst=arr[:, 1].copy(),
                 source=0, sink=len(labels) - 1, sites=sites)


# ----------------------------------------------------------------------------
# query generator


def _walk(g: Graph, rng: Rng, start_site: int, target: int, loop_reps: tuple) -> list[int]:
    """Vertices of a sub-walk from segment `start_site` until the spelled length reaches target."""
    lens = g.off
    walk: list[int] = []
    total = 0
    s = start_site
    sites = g.sites
    while s < len(sites):
        kind = sites[s][0]
        if kind == "seg":
            vs = [sites[s][1]]
        elif kind == "loop":
            reps = rng.one_int(*loop_reps)
            vs = [sites[s][1]] * reps
        else:
            alts, skippable = sites[s][1], sites[s][2]
            if skippable:
                vs = [alts[0]] if rng.one() < 0.5 else []
            else:
                vs = [alts[rng.one_int(0, len(alts) - 1)]]
        for v in vs:
            walk.append(v)
            total += int(lens[v + 1] - lens[v])
            if total >= target:
                return walk
        s += 1
    return walk


def _mutate(codes: np.ndarray, rate: float, weights: tuple, rng: Rng) -> tuple[np.ndarray, int]:
    """Single-base errors at per-base rate `rate`; weights = (sub, ins, del)."""
    n = len(codes)
    u = rng.uniform(n)
    t = rng.uniform(n)
    nb = rng.integers(0, 2, n).astype(np.uint8)   # substitute offset 1..3 - 1
    ib = rng.codes(n)
    err = u < rate
    w = np.asarray(weights, dtype=np.float64)
    w = np.cumsum(w / w.sum())
    typ = np.where(t < w[0], 0, np.where(t < w[1], 1, 2))
    sub = err & (typ == 0)
    ins = err & (typ == 1)
    dele = err & (typ == 2)
    out = codes.copy()
    out[sub] = (out[sub] + 1 + nb[sub]) & 3
    counts = np.where(dele, 0, np.where(ins, 2, 1))
    rep = np.repeat(out, counts)
    # for inserted positions, the second copy becomes the random inserted base
    ends = np.cumsum(counts) - 1
    ins_pos = ends[ins]
    rep[ins_pos] = ib[ins]
    return rep, int(err.sum())


def _codes_of(g: Graph, walk: list[int]) -> np.ndarray:
    parts = [g.seq[int(g.off[v]):int(g.off[v + 1])] for v in walk]
    asc = np.concatenate(parts) if parts else np.zeros(0, dtype=np.uint8)
    lut = np.zeros(256, dtype=np.uint8)
    lut[ord("C")] = 1
    lut[ord("G")] = 2
    lut[ord("T")] = 3
    return lut[asc]


def make_queries(g: Graph, n_queries: int, seed: int, length_fn, div_fn,
                 weights=(1, 1, 1), loop_reps=(1, 1), stream0: int = 1000) -> Queries:
    seg_idx = np.array([i for i, s in enumerate(g.sites) if s[0] == "seg"], dtype=np.int64)
    # spelled position of each site along the shortest allele choice, so that a start
    # segment can be drawn that leaves room for the whole walk
    glen = g.lengths()
    site_len = np.array([glen[s[1]] if s[0] != "alts" else
                         (0 if s[2] else min(glen[v] for v in s[1])) for s in g.sites],
                        dtype=np.int64)
    site_pos = np.concatenate([[0], np.cumsum(site_len)])
    total = int(site_pos[-1])
    seqs, vss, ves, eds, divs = [], [], [], [], []
    for qi in range(n_queries):
        rng = Rng(seed, stream0 + qi)
        target = int(length_fn(rng))
        div = float(div_fn(rng))
        room = seg_idx[site_pos[seg_idx] + target <= total]
        if len(room) == 0:
            room = seg_idx[:1]
        s0 = int(room[rng.one_int(0, len(room) - 1)])
        walk = _walk(g, rng, s0, target, loop_reps)
        codes = _codes_of(g, walk)
        mut, ned = _mutate(codes, div, weights, rng) if div > 0 else (codes, 0)
        seqs.append(_ACGT[mut])
        vss.append(walk[0])
        ves.append(walk[-1])
        eds.append(ned)
        divs.append(div)
    off = np.zeros(n_queries + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(s) for s in seqs])
    seq = np.concatenate(seqs) if seqs else np.zeros(0, dtype=np.uint8)
    return Queries(seq=seq, off=off, v_s=np.array(vss, dtype=np.uint32),
                   v_e=np.array(ves, dtype=np.uint32), edits=np.array(eds, dtype=np.int64),
                   divergence=np.array(divs, dtype=np.float64))


# ----------------------------------------------------------------------------
# the five workloads


def _loguniform(lo, hi):
    return lambda r: int(round(math.exp(math.log(lo) + r.one() * (math.log(hi) - math.log(lo)))))


def _lognormal(median, sigma, lo, hi):
    return lambda r: int(min(hi, max(lo, round(median * math.exp(sigma * float(r.normal(1)[0]))))))


def _uniform(lo, hi):
    return lambda r: lo + r.one() * (hi - lo)


def _const(x):
    return lambda r: x


CONFIGS = {
    # tiny: 2 kb backbone, a site every ~100 bp (70% SNP, 30% indel 1-10 bp);
    # 100 x 1 kb queries at 1% single-base errors (sub:ins:del = 1:1:1)
    1: dict(graph=GraphSpec(backbone=2000, gap=(50, 150), p_snp=0.7, p_indel=0.3, indel_len=(1, 10)),
            n=100, length=_const(1000), div=_const(0.01), weights=(1, 1, 1), loops=(1, 1)),
    # batched: 1 Mb backbone, a site every ~200 bp (SNP 70%, indel 1-50 25%, alt 200-2000 5%);
    # 10k queries, length log-uniform 1-20 kb, divergence U[0.5%, 5%]
    2: dict(graph=GraphSpec(backbone=1_000_000, gap=(100, 300), p_snp=0.7, p_indel=0.25,
                            indel_len=(1, 50), p_alt=0.05, alt_len=(200, 2000)),
            n=10_000, length=_loguniform(1000, 20000), div=_uniform(0.005, 0.05),
            weights=(1, 1, 1), loops=(1, 1)),
    # cyclic: config-2 graph plus a tandem-repeat loop (unit 2-200 bp) every 2.5-7.5 kb;
    # 2k x 50 kb queries, 8% errors, sub:ins:del = 2:5:3, loops taken 1-10 times
    3: dict(graph=GraphSpec(backbone=1_000_000, gap=(100, 300), p_snp=0.7, p_indel=0.25,
                            indel_len=(1, 50), p_alt=0.05, alt_len=(200, 2000),
                            loop_every=(2500, 7500), loop_unit=(2, 200)),
            n=2_000, length=_const(50_000), div=_const(0.08), weights=(2, 5, 3), loops=(1, 10)),
    # large: 50 Mb backbone with the config-2 site mix; 100k queries, lognormal length
    # (median 8 kb, sigma 0.8, clamped to 1-100 kb), divergence U[0.1%, 10%]
    4: dict(graph=GraphSpec(backbone=50_000_000, gap=(100, 300), p_snp=0.7, p_indel=0.25,
                            indel_len=(1, 50), p_alt=0.05, alt_len=(200, 2000)),
            n=100_000, length=_lognormal(8000, 0.8, 1000, 100_000), div=_uniform(0.001, 0.10),
            weights=(1, 1, 1), loops=(1, 1)),
}
CONFIGS[5] = dict(CONFIGS[4])


def make_config(cfg: int, n_queries: int | None = None, seed: int | None = None,
                backbone: int | None = None):
    """(graph, queries) for workload `cfg` (1..5); n_queries / backbone shrink it for tests."""
    c = CONFIGS[cfg]
    spec = c["graph"]
    if backbone is not None:
        spec = dataclasses.replace(spec, backbone=backbone)
    s = cfg if seed is None else seed
    g = make_graph(spec, s)
    n = c["n"] if n_queries is None else n_queries
    q = make_queries(g, n, s, c["length"], c["div"], c["weights"], c["loops"])
    return g, q


def poisson_arrivals(rate_per_s: float, duration_s: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process, for the serving workload."""
    rng = Rng(seed, 7)
    n_max = int(rate_per_s * duration_s * 1.5 + 64)
    gaps = -np.log(np.maximum(rng.uniform(n_max), 1e-300)) / rate_per_s
    t = np.cumsum(gaps)
    return t[t < duration_s]


def random_small_graph(rng: Rng, n_vertices: int, max_len: int, p_arc: float,
                       cyclic: bool) -> Graph:
    """Tiny random graph for brute-force pins: vertex i -> j arcs with probability p_arc
    (j > i only unless cyclic), plus a chain 0 -> 1 -> ... so the sink is reachable."""
    labels = []
    for _ in range(n_vertices):
        ln = rng.one_int(1, max_len)
        labels.append(_ACGT[rng.codes(ln)].tobytes())
    arcs = set()
    for i in range(n_vertices - 1):
        arcs.add((i, i + 1))
    for i in range(n_vertices):
        for j in range(n_vertices):
            if (j > i or cyclic) and rng.one() < p_arc:
                arcs.add((i, j))
    return Graph.from_lists(labels, sorted(arcs))
