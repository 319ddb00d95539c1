"""Pure-python brute-force pins for the oracle -- TEST INFRASTRUCTURE ONLY.

These are deliberately independent of oracle/gwfa_oracle.c: they enumerate
walks explicitly and use a textbook pairwise DP, so that a mistake in the C
oracle's recurrence (a dropped case of Eq. 1, a wrong index, an arc followed
the wrong way) shows up as a disagreement on tiny graphs.
"""
from __future__ import annotations

import heapq


def levenshtein_py(x: bytes, y: bytes) -> int:
    """Wagner-Fischer, full table."""
    n, m = len(x), len(y)
    D = [[0] * (m + 1) for _ in range(n + 1)]
    for a in range(n + 1):
        D[a][0] = a
    for b in range(m + 1):
        D[0][b] = b
    for a in range(1, n + 1):
        for b in range(1, m + 1):
            D[a][b] = min(D[a - 1][b] + 1, D[a][b - 1] + 1,
                          D[a - 1][b - 1] + (0 if x[a - 1] == y[b - 1] else 1))
    return D[n][m]


def best_walk_distance(labels: list[bytes], arcs: list[tuple[int, int]], q: bytes,
                       vs: int, ve: int, max_extra: int | None = None) -> int | None:
    """min over walks vs -> ve of d(sigma(w), q) (Def. 2), by enumerating walks.

    A walk whose spelled length L exceeds |q| + best has distance >= L - |q| > best,
    so the enumeration stops extending a walk once its length passes that bound;
    this keeps cyclic graphs finite and the answer exact.
    """
    succ: dict[int, list[int]] = {}
    for u, v in arcs:
        succ.setdefault(u, []).append(v)
    best = [None]
    bound = len(q) + (max_extra if max_extra is not None else len(q) + sum(len(x) for x in labels))

    def rec(v: int, spelled: bytes):
        s = spelled + labels[v]
        lim = bound if best[0] is None else min(bound, len(q) + best[0])
        if len(s) > lim:
            return
        if v == ve:
            d = levenshtein_py(s, q)
            if best[0] is None or d < best[0]:
                best[0] = d
        for u in succ.get(v, []):
            rec(u, s)

    rec(vs, b"")
    return best[0]


def shortest_spelled_walk(labels: list[bytes], arcs: list[tuple[int, int]], vs: int,
                          ve: int) -> int | None:
    """Dijkstra with vertex weights |v|: length of the shortest spelled vs -> ve walk."""
    succ: dict[int, list[int]] = {}
    for u, v in arcs:
        succ.setdefault(u, []).append(v)
    dist = {vs: len(labels[vs])}
    pq = [(len(labels[vs]), vs)]
    while pq:
        d, v = heapq.heappop(pq)
        if d > dist.get(v, 1 << 60):
            continue
        if v == ve:
            return d
        for u in succ.get(v, []):
            nd = d + len(labels[u])
            if nd < dist.get(u, 1 << 60):
                dist[u] = nd
                heapq.heappush(pq, (nd, u))
    return None


def best_walk_distance_ends(labels: list[bytes], arcs: list[tuple[int, int]], q: bytes, vs: int,
                            ve: int, free_start: bool, free_end: bool, extend: bool) -> int | None:
    """The formulation variants of Sec. 2.1 by enumeration: min over walks w from vs
    (ending at ve, or anywhere when `extend`) and over the prefix a of sigma(vs) the
    walk may skip (free_start) and the suffix b of its last vertex it may skip
    (free_end or extend) of d(sigma(w)[a : |sigma(w)| - b], q).

    Any walk that extends w by a vertex u aligns a segment of at least
    |sigma(w)| - a >= |sigma(w)| - |vs| bases (only u's own bases may be skipped at
    the end), so once |sigma(w)| - |vs| exceeds |q| + best no extension of w can
    improve on best.
    """
    succ: dict[int, list[int]] = {}
    for u, v in arcs:
        succ.setdefault(u, []).append(v)
    best = [None]
    skip0 = len(labels[vs]) if free_start else 0
    cap = 2 * len(q) + sum(len(x) for x in labels) + skip0   # before any walk qualifies

    def rec(v: int, spelled: bytes):
        s = spelled + labels[v]
        if extend or v == ve:
            starts = range(len(labels[vs]) + 1) if free_start else [0]
            ends = range(len(labels[v]) + 1) if (free_end or extend) else [0]
            for a in starts:
                for b in ends:
                    if a > len(s) - b:
                        continue
                    d = levenshtein_py(s[a:len(s) - b], q)
                    if best[0] is None or d < best[0]:
                        best[0] = d
        lim = cap if best[0] is None else len(q) + best[0]
        if len(s) - skip0 > lim:
            return
        for u in succ.get(v, []):
            rec(u, s)

    rec(vs, b"")
    return best[0]
