/*
 * gwfa_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * The CPU oracle for the graph wavefront alignment library.  Only the test
 * suite, the package smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, table or helper with the CUDA path: it reads
 * the graph as ASCII labels plus an arc list, exactly as a user would hand it
 * to the library, and computes everything itself in plain, slow C.
 *
 * Functions (each cites the passage it follows):
 *
 *   oracle_levenshtein  textbook unit-cost edit distance (Sec. 2.1, d(x, y)).
 *   oracle_dp           Eq. 1: the cell recurrence H_{i,v,j} over a
 *                       string-labelled graph, initial condition H_{0,vs,0}=0,
 *                       answer H_{|q|,ve,|ve|} (Sec. 2.2).  This is the
 *                       definition of the optimal global distance (Def. 2).
 *   oracle_gwfa         Alg. 1 (GwfEditDist) driving Alg. 2 (GwfExtend),
 *                       Alg. 3 (GwfExpand) and, when a_diff > 0, Alg. 4
 *                       (GwfPrune), in the paper's order, single threaded, with
 *                       a FIFO queue.  It is the reference for pruned distances
 *                       and for the work counts (sum and peak of |Q|).
 *   oracle_dp_ends,     the same two with the formulation variants Sec. 2.1
 *   oracle_gwfa_ends    mentions (their details are in a supplement that is not
 *                       available; these are read off Eq. 1 and Alg. 1):
 *                         OR_FREE_START  the walk may begin at any position of
 *                                        v_s: row 0 of Eq. 1 is 0 on every cell
 *                                        of v_s; Alg. 1 starts from the
 *                                        diagonals (v_s, -j) with offset j;
 *                         OR_FREE_END    the walk may end at any position of
 *                                        v_e: the answer is min_j H_{|q|,ve,j};
 *                                        Alg. 1 stops at the first score whose
 *                                        extension puts a diagonal of v_e on
 *                                        query position |q|;
 *                         OR_EXTEND      no end vertex: the whole query is
 *                                        aligned to a walk from v_s that ends
 *                                        anywhere: min over v, j of H_{|q|,v,j};
 *                                        Alg. 1 stops when any diagonal reaches
 *                                        query position |q|.
 *                       A walk may skip a whole end vertex (j = 0 at v_e is the
 *                       end of a predecessor).  Pruning is not combined with
 *                       the variants.
 *
 * Readings of points the paper leaves open (they are the library's readings
 * too, stated once more here so this file stands alone):
 *   - Strings are 1-based in the paper; here q[i] of the paper is q[i-1].
 *   - The set H~ persists across scores: an entry is only ever overwritten by
 *     Alg. 3's write-back (or Alg. 2's extension of that same diagonal), never
 *     removed, and a pruned diagonal keeps its offset (Alg. 4 writes back only
 *     the survivors).
 *   - W~ (aligned graph walk length, Alg. 4) is base + H~ where base is the
 *     spelled length of the walk before vertex v: base(vs,0) = 0, a spill
 *     across arc (v,u) gives base(v,k) + |v|, an expansion candidate keeps the
 *     base of the diagonal it came from.  Ties: Alg. 3's max-merge compares
 *     (offset, base) lexicographically; in Alg. 2 a diagonal that is absent
 *     when spilled into takes the largest base among the spills of the same
 *     FIFO generation (the FIFO queue of Alg. 2 is breadth first: generation
 *     g+1 is everything pushed while generation g is popped); a diagonal that
 *     was present before that generation is never changed by a spill.
 *   - Alg. 4 runs after d <- d+1 and before Expand, every score.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_INF INT32_MAX

/* status codes returned by the oracle (negative = no distance) */
#define OR_OK 0
#define OR_ERR_INVALID (-1)
#define OR_ERR_UNREACHABLE (-4)
#define OR_ERR_EMPTY_FRONTIER (-5)
#define OR_ERR_SCORE_LIMIT (-8)
#define OR_ERR_OOM (-2)

/* formulation variants (flags) */
#define OR_FREE_START 1
#define OR_FREE_END 2
#define OR_EXTEND 4

static int code_of(char c) {
    switch (c) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    default: return -1;
    }
}

/* --------------------------------------------------------------------------
 * Levenshtein distance: D[a][b] = min(D[a-1][b]+1, D[a][b-1]+1,
 * D[a-1][b-1] + [x_a != y_b]), D[a][0] = a, D[0][b] = b.  Two rows.
 */
int64_t oracle_levenshtein(const char *x, uint64_t nx, const char *y, uint64_t ny) {
    int64_t *prev = (int64_t *)malloc((ny + 1) * sizeof(int64_t));
    int64_t *cur = (int64_t *)malloc((ny + 1) * sizeof(int64_t));
    if (!prev || !cur) { free(prev); free(cur); return OR_ERR_OOM; }
    for (uint64_t b = 0; b <= ny; ++b) prev[b] = (int64_t)b;
    for (uint64_t a = 1; a <= nx; ++a) {
        cur[0] = (int64_t)a;
        for (uint64_t b = 1; b <= ny; ++b) {
            int64_t best = prev[b] + 1;
            if (cur[b - 1] + 1 < best) best = cur[b - 1] + 1;
            int64_t diag = prev[b - 1] + (code_of(x[a - 1]) != code_of(y[b - 1]) ? 1 : 0);
            if (diag < best) best = diag;
            cur[b] = best;
        }
        int64_t *t = prev; prev = cur; cur = t;
    }
    int64_t r = prev[ny];
    free(prev); free(cur);
    return r;
}

/* --------------------------------------------------------------------------
 * Graph as the oracle sees it: labels decoded to codes 0..3, plus forward and
 * reverse adjacency built from the arc list (duplicates kept; they are harmless
 * to both algorithms).
 */
typedef struct {
    uint32_t nv;
    uint8_t *lab;       /* all labels as codes */
    uint64_t *off;      /* nv+1 */
    uint32_t *out_off, *out_dst;   /* CSR of out-arcs */
    uint32_t *in_off, *in_src;     /* CSR of in-arcs */
    int forward_ids;    /* 1 if every arc u->v has u < v or u == v */
} og_graph;

static void og_free(og_graph *g) {
    free(g->lab); free(g->off); free(g->out_off); free(g->out_dst);
    free(g->in_off); free(g->in_src);
}

static int og_build(og_graph *g, uint32_t nv, const char *seq, const uint64_t *seq_off,
                    uint64_t na, const uint32_t *asrc, const uint32_t *adst) {
    memset(g, 0, sizeof(*g));
    g->nv = nv;
    uint64_t tot = seq_off[nv];
    g->lab = (uint8_t *)malloc(tot ? tot : 1);
    g->off = (uint64_t *)malloc((nv + 1) * sizeof(uint64_t));
    g->out_off = (uint32_t *)calloc(nv + 1, sizeof(uint32_t));
    g->in_off = (uint32_t *)calloc(nv + 1, sizeof(uint32_t));
    g->out_dst = (uint32_t *)malloc((na ? na : 1) * sizeof(uint32_t));
    g->in_src = (uint32_t *)malloc((na ? na : 1) * sizeof(uint32_t));
    if (!g->lab || !g->off || !g->out_off || !g->in_off || !g->out_dst || !g->in_src) {
        og_free(g); return OR_ERR_OOM;
    }
    for (uint32_t v = 0; v <= nv; ++v) g->off[v] = seq_off[v] - seq_off[0];
    for (uint32_t v = 0; v < nv; ++v) {
        if (seq_off[v + 1] <= seq_off[v]) { og_free(g); return OR_ERR_INVALID; }
    }
    for (uint64_t p = 0; p < tot; ++p) {
        int c = code_of(seq[seq_off[0] + p]);
        if (c < 0) { og_free(g); return OR_ERR_INVALID; }
        g->lab[p] = (uint8_t)c;
    }
    g->forward_ids = 1;
    for (uint64_t a = 0; a < na; ++a) {
        if (asrc[a] >= nv || adst[a] >= nv) { og_free(g); return OR_ERR_INVALID; }
        g->out_off[asrc[a] + 1]++;
        g->in_off[adst[a] + 1]++;
        if (asrc[a] > adst[a]) g->forward_ids = 0;
    }
    for (uint32_t v = 0; v < nv; ++v) {
        g->out_off[v + 1] += g->out_off[v];
        g->in_off[v + 1] += g->in_off[v];
    }
    uint32_t *fo = (uint32_t *)malloc((nv + 1) * sizeof(uint32_t));
    uint32_t *fi = (uint32_t *)malloc((nv + 1) * sizeof(uint32_t));
    if (!fo || !fi) { free(fo); free(fi); og_free(g); return OR_ERR_OOM; }
    memcpy(fo, g->out_off, (nv + 1) * sizeof(uint32_t));
    memcpy(fi, g->in_off, (nv + 1) * sizeof(uint32_t));
    for (uint64_t a = 0; a < na; ++a) {
        g->out_dst[fo[asrc[a]]++] = adst[a];
        g->in_src[fi[adst[a]]++] = asrc[a];
    }
    free(fo); free(fi);
    return OR_OK;
}

static inline uint32_t og_len(const og_graph *g, uint32_t v) {
    return (uint32_t)(g->off[v + 1] - g->off[v]);
}

/* breadth-first reachability along out-arcs (dir=0) or in-arcs (dir=1) */
static uint8_t *og_reach(const og_graph *g, uint32_t from, int dir) {
    uint8_t *seen = (uint8_t *)calloc(g->nv, 1);
    uint32_t *stack = (uint32_t *)malloc((g->nv + 1) * sizeof(uint32_t));
    if (!seen || !stack) { free(seen); free(stack); return NULL; }
    uint32_t top = 0;
    seen[from] = 1; stack[top++] = from;
    while (top) {
        uint32_t v = stack[--top];
        const uint32_t *o = dir ? g->in_off : g->out_off;
        const uint32_t *n = dir ? g->in_src : g->out_dst;
        for (uint32_t a = o[v]; a < o[v + 1]; ++a) {
            uint32_t u = n[a];
            if (!seen[u]) { seen[u] = 1; stack[top++] = u; }
        }
    }
    free(stack);
    return seen;
}

/* --------------------------------------------------------------------------
 * oracle_dp: Eq. 1.
 *
 *   H_{i,v,j} = min( H_{i-1,v,j} + 1                      (i >= 1)
 *                    H_{i,v,j-1} + 1                      (j >= 1)
 *                    H_{i-1,v,j-1} + Delta_{i,v,j}        (i, j >= 1)
 *                    H_{i,u,|u|}  for every arc (u, v)    (j == 0) )
 *   H_{0,vs,0} = 0, every other cell without an applicable case is infinite,
 *   answer H_{|q|,ve,|ve|}.
 *
 * Only vertices on some vs->ve walk can carry a cell that feeds the answer, so
 * the table is restricted to S = {v : vs reaches v and v reaches ve} (exact:
 * every walk from vs to ve lies in S).  Row i is computed from row i-1 in two
 * steps: first the two cases that read row i-1 (the candidates c), then the
 * two cases inside row i, which form a shortest-path closure along the graph
 * (cost 1 per step inside a vertex, cost 0 across an arc).  Every cycle of that
 * closure passes through whole vertices of length >= 1, so its fixpoint is
 * unique and is reached by Gauss-Seidel sweeps in vertex-id order repeated
 * until nothing changes; a self arc is resolved on the spot by repeating that
 * vertex until it is stable.  When the ids are a topological order apart from
 * self arcs, the first sweep is already the fixpoint.
 */
static int dp_relax_vertex(const og_graph *g, const uint8_t *inS, uint32_t v,
                           int32_t *row, const uint64_t *col, int self_loop) {
    /* row[col[v]+j], j = 0..|v|; the candidates c are already stored there */
    int changed = 0;
    uint32_t lv = og_len(g, v);
    int32_t *h = row + col[v];
    for (;;) {   /* values only decrease; a self arc settles within two passes */
        int32_t h0 = h[0];
        for (uint32_t a = g->in_off[v]; a < g->in_off[v + 1]; ++a) {
            uint32_t u = g->in_src[a];
            if (!inS[u]) continue;
            int32_t hu = row[col[u] + og_len(g, u)];
            if (hu < h0) h0 = hu;
        }
        int local = 0;
        if (h0 < h[0]) { h[0] = h0; local = 1; }
        for (uint32_t j = 1; j <= lv; ++j) {
            if (h[j - 1] != OR_INF && h[j - 1] + 1 < h[j]) { h[j] = h[j - 1] + 1; local = 1; }
        }
        changed |= local;
        if (!self_loop || !local) break;
    }
    return changed;
}

int64_t oracle_dp_ends(uint32_t nv, const char *seq, const uint64_t *seq_off,
                       uint64_t na, const uint32_t *asrc, const uint32_t *adst,
                       const char *q, uint64_t n, uint32_t vs, uint32_t ve, int ends) {
    og_graph g;
    if (ends & ~(OR_FREE_START | OR_FREE_END | OR_EXTEND)) return OR_ERR_INVALID;
    const int extend = (ends & OR_EXTEND) != 0;
    int st = og_build(&g, nv, seq, seq_off, na, asrc, adst);
    if (st) return st;
    if (extend) ve = vs;   /* no end vertex */
    if (vs >= nv || ve >= nv) { og_free(&g); return OR_ERR_INVALID; }
    uint8_t *qc = (uint8_t *)malloc(n ? n : 1);
    for (uint64_t i = 0; i < n; ++i) {
        int c = code_of(q[i]);
        if (c < 0) { free(qc); og_free(&g); return OR_ERR_INVALID; }
        qc[i] = (uint8_t)c;
    }
    uint8_t *fw = og_reach(&g, vs, 0), *bw = og_reach(&g, ve, 1);
    if (!fw || !bw) { free(fw); free(bw); free(qc); og_free(&g); return OR_ERR_OOM; }
    if (!fw[ve]) { free(fw); free(bw); free(qc); og_free(&g); return OR_ERR_UNREACHABLE; }
    uint8_t *inS = fw;
    uint32_t nS = 0;
    /* S: the vertices on some vs->ve walk; without an end vertex, all reachable ones */
    for (uint32_t v = 0; v < nv; ++v) { inS[v] = fw[v] && (extend || bw[v]); nS += inS[v]; }
    free(bw);
    uint32_t *Sv = (uint32_t *)malloc((nS ? nS : 1) * sizeof(uint32_t));
    uint8_t *selfl = (uint8_t *)calloc(nv, 1);
    uint64_t *col = (uint64_t *)malloc(nv * sizeof(uint64_t));
    uint64_t ncol = 0;
    uint32_t t = 0;
    int one_sweep = g.forward_ids;
    for (uint32_t v = 0; v < nv; ++v) {
        if (!inS[v]) continue;
        Sv[t++] = v;
        col[v] = ncol;
        ncol += og_len(&g, v) + 1;
        for (uint32_t a = g.out_off[v]; a < g.out_off[v + 1]; ++a)
            if (g.out_dst[a] == v) selfl[v] = 1;
    }
    int32_t *prev = (int32_t *)malloc(ncol * sizeof(int32_t));
    int32_t *cur = (int32_t *)malloc(ncol * sizeof(int32_t));
    if (!Sv || !col || !prev || !cur || !selfl) {
        free(Sv); free(col); free(prev); free(cur); free(selfl); free(inS); free(qc); og_free(&g);
        return OR_ERR_OOM;
    }
    /* row 0: only the initial condition and the in-row cases */
    for (uint64_t c = 0; c < ncol; ++c) prev[c] = OR_INF;
    prev[col[vs]] = 0;
    if (ends & OR_FREE_START)   /* the walk may begin at any position of vs */
        for (uint32_t j = 0; j <= og_len(&g, vs); ++j) prev[col[vs] + j] = 0;
    for (;;) {
        int ch = 0;
        for (uint32_t s = 0; s < nS; ++s) ch |= dp_relax_vertex(&g, inS, Sv[s], prev, col, selfl[Sv[s]]);
        if (one_sweep || !ch) break;
    }
    for (uint64_t i = 1; i <= n; ++i) {
        uint8_t qi = qc[i - 1];
        for (uint32_t s = 0; s < nS; ++s) {
            uint32_t v = Sv[s];
            uint32_t lv = og_len(&g, v);
            const uint8_t *lab = g.lab + g.off[v];
            const int32_t *hp = prev + col[v];
            int32_t *hc = cur + col[v];
            /* case 1 (insertion) for every j; case 3 (diagonal) for j >= 1 */
            hc[0] = hp[0] == OR_INF ? OR_INF : hp[0] + 1;
            for (uint32_t j = 1; j <= lv; ++j) {
                int32_t best = hp[j] == OR_INF ? OR_INF : hp[j] + 1;
                if (hp[j - 1] != OR_INF) {
                    int32_t dg = hp[j - 1] + (lab[j - 1] != qi ? 1 : 0);
                    if (dg < best) best = dg;
                }
                hc[j] = best;
            }
        }
        /* cases 2 and 4: closure inside row i */
        for (;;) {
            int ch = 0;
            for (uint32_t s = 0; s < nS; ++s) ch |= dp_relax_vertex(&g, inS, Sv[s], cur, col, selfl[Sv[s]]);
            if (one_sweep || !ch) break;
        }
        int32_t *tt = prev; prev = cur; cur = tt;
    }
    int64_t ans = prev[col[ve] + og_len(&g, ve)];
    if (extend) {                         /* min over every cell of row |q| */
        for (uint64_t c = 0; c < ncol; ++c) if (prev[c] < ans) ans = prev[c];
    } else if (ends & OR_FREE_END) {      /* min over the cells of ve in row |q| */
        for (uint32_t j = 0; j <= og_len(&g, ve); ++j)
            if (prev[col[ve] + j] < ans) ans = prev[col[ve] + j];
    }
    free(Sv); free(col); free(prev); free(cur); free(selfl); free(inS); free(qc); og_free(&g);
    return ans == OR_INF ? OR_ERR_UNREACHABLE : ans;
}

int64_t oracle_dp(uint32_t nv, const char *seq, const uint64_t *seq_off,
                  uint64_t na, const uint32_t *asrc, const uint32_t *adst,
                  const char *q, uint64_t n, uint32_t vs, uint32_t ve) {
    return oracle_dp_ends(nv, seq, seq_off, na, asrc, adst, q, n, vs, ve, 0);
}

/* --------------------------------------------------------------------------
 * oracle_gwfa: Alg. 1-4.
 *
 * The graph wavefront set H~ maps a diagonal (v, k) to its furthest offset j
 * (plus the walk base used by W~).  It is a plain open-addressing hash map.
 */
typedef struct {
    uint64_t key;      /* (v << 32) | (uint32_t)k; EMPTY_KEY when unused */
    int32_t j;         /* H~_{v,k} */
    int64_t base;      /* W~_{v,k} - H~_{v,k} */
    uint64_t spill_mark;  /* (extend call << 20) | generation at which a spill inserted it */
} ent_t;

#define EMPTY_KEY UINT64_MAX

typedef struct {
    ent_t *e;
    uint64_t cap, n;
} hmap;

static inline uint64_t dkey(uint32_t v, int32_t k) { return ((uint64_t)v << 32) | (uint32_t)k; }

static inline uint64_t hmix(uint64_t x) {
    x ^= x >> 33; x *= 0xff51afd7ed558ccdULL; x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ULL; x ^= x >> 33;
    return x;
}

static int hm_init(hmap *m, uint64_t cap) {
    m->cap = cap; m->n = 0;
    m->e = (ent_t *)malloc(cap * sizeof(ent_t));
    if (!m->e) return OR_ERR_OOM;
    for (uint64_t i = 0; i < cap; ++i) m->e[i].key = EMPTY_KEY;
    return OR_OK;
}

static ent_t *hm_find(const hmap *m, uint64_t key) {
    uint64_t h = hmix(key) & (m->cap - 1);
    for (;;) {
        if (m->e[h].key == key) return &m->e[h];
        if (m->e[h].key == EMPTY_KEY) return NULL;
        h = (h + 1) & (m->cap - 1);
    }
}

static ent_t *hm_insert(hmap *m, uint64_t key);

static int hm_grow(hmap *m) {
    hmap n2;
    if (hm_init(&n2, m->cap * 2)) return OR_ERR_OOM;
    for (uint64_t i = 0; i < m->cap; ++i) {
        if (m->e[i].key == EMPTY_KEY) continue;
        ent_t *d = hm_insert(&n2, m->e[i].key);
        *d = m->e[i];
    }
    free(m->e);
    *m = n2;
    return OR_OK;
}

/* returns the entry for key, inserting an uninitialised one if absent
 * (the caller checks presence with hm_find first) */
static ent_t *hm_insert(hmap *m, uint64_t key) {
    if ((m->n + 1) * 2 > m->cap) { if (hm_grow(m)) return NULL; }
    uint64_t h = hmix(key) & (m->cap - 1);
    while (m->e[h].key != EMPTY_KEY && m->e[h].key != key) h = (h + 1) & (m->cap - 1);
    if (m->e[h].key == EMPTY_KEY) { m->e[h].key = key; m->n++; }
    return &m->e[h];
}

static void hm_clear(hmap *m) {
    for (uint64_t i = 0; i < m->cap; ++i) m->e[i].key = EMPTY_KEY;
    m->n = 0;
}

typedef struct { uint32_t v; int32_t k; } diag_t;

typedef struct {
    diag_t *a;
    uint64_t n, cap;
} dvec;

static int dv_push(dvec *q, uint32_t v, int32_t k) {
    if (q->n == q->cap) {
        uint64_t nc = q->cap ? q->cap * 2 : 1024;
        diag_t *na = (diag_t *)realloc(q->a, nc * sizeof(diag_t));
        if (!na) return OR_ERR_OOM;
        q->a = na; q->cap = nc;
    }
    q->a[q->n].v = v; q->a[q->n].k = k; q->n++;
    return OR_OK;
}

/* result record, filled by oracle_gwfa (layout mirrored by the python wrapper) */
typedef struct {
    int64_t distance;      /* d, or a negative status */
    int64_t is_upper_bound;/* 1 iff pruning dropped at least one diagonal */
    int64_t n_scores;      /* number of GwfExtend calls = d + 1 on success */
    int64_t cells;         /* sum over scores of |Q| after GwfExtend */
    int64_t peak;          /* max over scores of |Q| after GwfExtend */
    int64_t visited;       /* insertions into H~ (= distinct diagonals ever inserted
                              unless eviction removed some and they came back) */
    int64_t pruned;        /* diagonals dropped by GwfPrune, summed over scores */
    int64_t spills;        /* diagonals inserted by GwfExtend's arc loop */
    int64_t evicted;       /* entries removed from H~ by the memory bound (evict_lag) */
} oracle_stats;

/* LCP(q[i+1..|q|], v[j+1..|v|]) in the paper's 1-based notation */
static inline int64_t lcp(const uint8_t *q, int64_t n, int64_t i, const uint8_t *lab, int64_t lv,
                          int64_t j) {
    int64_t l = 0;
    while (i + l < n && j + l < lv && q[i + l] == lab[j + l]) ++l;
    return l;
}

/* Memory-bounded H~ (with pruning only): every evict_every scores, right after
 * GwfExpand, the entries that are not in the new Q and whose anti-diagonal
 * a = i + W~ (Alg. 4's measure) lags this score's a_max by evict_lag or more are
 * removed from H~.  A removed diagonal may be inserted again later (it counts as a
 * new insertion); every offset is still that of a realised alignment, so the
 * distance stays an upper bound of the exact one. */
#define KEEP_MARK (UINT64_MAX - 1)

/* The removal step itself: keep the entries of `keep` (the new Q) and those whose
 * a = i + W~ lags amax by less than lag (or by at most lag, with the planted `le`
 * mistake); count the others in out->evicted. */
static int evict(hmap *H, const dvec *keep, int64_t amax, int64_t lag, int le, oracle_stats *out) {
    for (uint64_t p = 0; p < keep->n; ++p) hm_find(H, dkey(keep->a[p].v, keep->a[p].k))->spill_mark = KEEP_MARK;
    hmap H2 = {0};
    if (hm_init(&H2, H->cap)) return OR_ERR_OOM;
    for (uint64_t x = 0; x < H->cap; ++x) {
        ent_t *e = &H->e[x];
        if (e->key == EMPTY_KEY) continue;
        int64_t k = (int32_t)(uint32_t)(e->key & 0xFFFFFFFFu);
        int64_t a = (k + e->j) + (e->base + e->j);   /* i + W~ */
        if (e->spill_mark == KEEP_MARK || amax - a < lag || (le && amax - a == lag)) {
            ent_t *c = hm_insert(&H2, e->key);
            if (!c) { free(H2.e); return OR_ERR_OOM; }
            *c = *e;
            c->spill_mark = UINT64_MAX;
        } else {
            out->evicted++;
        }
    }
    free(H->e);
    *H = H2;
    return OR_OK;
}

int oracle_gwfa_ex(uint32_t nv, const char *seq, const uint64_t *seq_off,
                   uint64_t na, const uint32_t *asrc, const uint32_t *adst,
                   const char *qs, uint64_t n, uint32_t vs, uint32_t ve,
                   int64_t a_diff, int64_t max_score, int ends, int64_t evict_lag, int64_t evict_every,
                   oracle_stats *out) {
    memset(out, 0, sizeof(*out));
    og_graph g;
    if ((ends & ~(OR_FREE_START | OR_FREE_END | OR_EXTEND)) || (ends && a_diff > 0) ||
        evict_lag < 0 || (evict_lag > 0 && (a_diff <= 0 || evict_every <= 0))) {
        out->distance = OR_ERR_INVALID;
        return OR_ERR_INVALID;
    }
    const int extend = (ends & OR_EXTEND) != 0;
    /* a planted mistake for the tests only: same-generation spills keep the first
       base instead of the largest, which makes the result depend on the arc order */
    const int plant_first_tie = getenv("GWFA_ORACLE_PLANT_FIRST_TIE") != NULL;
    /* planted mistakes in the memory bound, for the tests only (each must change a
       hand-traced counter): keep an entry lagging by exactly evict_lag; keep by Q as
       GwfExtend left it instead of the new Q; evict before GwfExpand instead of after */
    const int plant_evict_le = getenv("GWFA_ORACLE_PLANT_EVICT_LE") != NULL;
    const int plant_evict_oldq = getenv("GWFA_ORACLE_PLANT_EVICT_OLDQ") != NULL;
    const int plant_evict_before = getenv("GWFA_ORACLE_PLANT_EVICT_BEFORE") != NULL;
    int st = og_build(&g, nv, seq, seq_off, na, asrc, adst);
    if (st) { out->distance = st; return st; }
    if (extend) ve = vs;   /* no end vertex */
    if (vs >= nv || ve >= nv) { og_free(&g); out->distance = OR_ERR_INVALID; return OR_ERR_INVALID; }
    uint8_t *q = (uint8_t *)malloc(n ? n : 1);
    for (uint64_t i = 0; i < n; ++i) {
        int c = code_of(qs[i]);
        if (c < 0) { free(q); og_free(&g); out->distance = OR_ERR_INVALID; return OR_ERR_INVALID; }
        q[i] = (uint8_t)c;
    }
    /* the paper assumes ve is reachable (Sec. 2.4); otherwise the loop would not end */
    uint8_t *fw = og_reach(&g, vs, 0);
    if (!fw) { free(q); og_free(&g); out->distance = OR_ERR_OOM; return OR_ERR_OOM; }
    int reach = fw[ve];
    free(fw);
    if (!reach) { free(q); og_free(&g); out->distance = OR_ERR_UNREACHABLE; return OR_ERR_UNREACHABLE; }

    hmap H = {0}, Hp = {0};
    int64_t inserted = 0;   /* insertions into H~ */
    dvec Q = {0}, Qp = {0}, Qx = {0};
    int rc = OR_OK;
    if (hm_init(&H, 1 << 12) || hm_init(&Hp, 1 << 12)) { rc = OR_ERR_OOM; goto done; }

    /* Alg. 1 */
    int64_t ke = (int64_t)n - og_len(&g, ve);        /* k_e <- |q| - |v_e| */
    {
        ent_t *e0 = hm_insert(&H, dkey(vs, 0));     /* H~_{v_s,0} <- 0 */
        ++inserted;
        e0->j = 0; e0->base = 0; e0->spill_mark = UINT64_MAX;
    }
    if (dv_push(&Q, vs, 0)) { rc = OR_ERR_OOM; goto done; }  /* Q <- [(v_s, 0)] */
    if (ends & OR_FREE_START) {   /* query position 0 against every position j of vs */
        for (int32_t j = 1; j <= (int32_t)og_len(&g, vs); ++j) {
            ent_t *e = hm_insert(&H, dkey(vs, -j));   /* H~_{v_s,-j} <- j */
            if (!e) { rc = OR_ERR_OOM; goto done; }
            ++inserted;
            e->j = j; e->base = 0; e->spill_mark = UINT64_MAX;
            if (dv_push(&Q, vs, -j)) { rc = OR_ERR_OOM; goto done; }
        }
    }
    int64_t d = 0;                                    /* d <- 0 */
    uint64_t ext_call = 0;
    for (;;) {
        /* ---- GwfExtend (Alg. 2) ---- */
        ++ext_call;
        Qp.n = 0;
        uint64_t head = 0, gen_end = Q.n, gen = 0;
        while (head < Q.n) {
            if (head == gen_end) { ++gen; gen_end = Q.n; }
            diag_t x = Q.a[head++];                   /* (v,k) <- Q.pop() */
            ent_t *e = hm_find(&H, dkey(x.v, x.k));
            int64_t j = e->j;                         /* j <- H~_{v,k} */
            int64_t i = x.k + j;                      /* i <- k + j */
            uint32_t lv = og_len(&g, x.v);
            int64_t l = lcp(q, (int64_t)n, i, g.lab + g.off[x.v], lv, j);
            e->j = (int32_t)(j + l);                  /* H~_{v,k} <- j + l */
            e->spill_mark = UINT64_MAX;
            int64_t base = e->base;
            if (dv_push(&Qp, x.v, x.k)) { rc = OR_ERR_OOM; goto done; }  /* Q'.push(v,k) */
            if (j + l == lv) {                        /* H~_{v,k} = |v| */
                for (uint32_t a = g.out_off[x.v]; a < g.out_off[x.v + 1]; ++a) {
                    uint32_t u = g.out_dst[a];
                    int32_t ku = x.k + (int32_t)lv;
                    ent_t *t = hm_find(&H, dkey(u, ku));
                    uint64_t mark = (ext_call << 20) | (gen + 1);
                    if (!t) {                         /* H~_{u,k+|v|} not in H~ */
                        t = hm_insert(&H, dkey(u, ku));
                        if (!t) { rc = OR_ERR_OOM; goto done; }
                        ++inserted;
                        t->j = 0;                     /* H~_{u,k+|v|} <- 0 */
                        t->base = base + lv;
                        t->spill_mark = mark;
                        out->spills++;
                        if (dv_push(&Q, u, ku)) { rc = OR_ERR_OOM; goto done; }  /* Q.push */
                    } else if (t->spill_mark == mark && base + lv > t->base && !plant_first_tie) {
                        t->base = base + lv;          /* same-generation tie: larger base */
                    }
                }
            }
        }
        { dvec tq = Q; Q = Qp; Qp = tq; }            /* Q <- Q' */
        out->n_scores++;
        out->cells += (int64_t)Q.n;
        if ((int64_t)Q.n > out->peak) out->peak = (int64_t)Q.n;

        /* end test of Alg. 1 */
        ent_t *ee = hm_find(&H, dkey(ve, (int32_t)ke));
        if (ee && ee->j == (int32_t)og_len(&g, ve)) break;
        if (ends & (OR_FREE_END | OR_EXTEND)) {   /* a diagonal just extended reached |q| */
            int hit = 0;
            for (uint64_t p = 0; p < Q.n && !hit; ++p) {
                if (!extend && Q.a[p].v != ve) continue;
                ent_t *e = hm_find(&H, dkey(Q.a[p].v, Q.a[p].k));
                hit = (int64_t)Q.a[p].k + e->j == (int64_t)n;
            }
            if (hit) break;
        }
        if (max_score >= 0 && d >= max_score) { rc = OR_ERR_SCORE_LIMIT; goto done; }
        d = d + 1;                                    /* d <- d + 1 */

        if (plant_evict_oldq) {                     /* planted mistake: remember Q after GwfExtend */
            Qx.n = 0;
            for (uint64_t p = 0; p < Q.n; ++p)
                if (dv_push(&Qx, Q.a[p].v, Q.a[p].k)) { rc = OR_ERR_OOM; goto done; }
        }

        /* ---- GwfPrune (Alg. 4), between d <- d+1 and GwfExpand ---- */
        int64_t amax = 0;
        if (a_diff > 0) {
            for (uint64_t p = 0; p < Q.n; ++p) {
                ent_t *e = hm_find(&H, dkey(Q.a[p].v, Q.a[p].k));
                int64_t i = Q.a[p].k + (int64_t)e->j;
                int64_t a = i + (e->base + e->j);     /* a <- i + W~_{v,k} */
                if (a > amax) amax = a;
            }
            if (amax > a_diff) {
                Qp.n = 0;
                for (uint64_t p = 0; p < Q.n; ++p) {
                    ent_t *e = hm_find(&H, dkey(Q.a[p].v, Q.a[p].k));
                    int64_t i = Q.a[p].k + (int64_t)e->j;
                    int64_t a = i + (e->base + e->j);
                    if (amax - a < a_diff) {          /* keep; its H~ is unchanged */
                        if (dv_push(&Qp, Q.a[p].v, Q.a[p].k)) { rc = OR_ERR_OOM; goto done; }
                    }
                }
                if (Qp.n < Q.n) { out->is_upper_bound = 1; out->pruned += (int64_t)(Q.n - Qp.n); }
                dvec tq = Q; Q = Qp; Qp = tq;
            }
        }

        if (evict_lag > 0 && d % evict_every == 0 && plant_evict_before) {   /* planted mistake */
            rc = evict(&H, &Q, amax, evict_lag, plant_evict_le, out);
            if (rc) goto done;
        }

        /* ---- GwfExpand (Alg. 3) ---- */
        hm_clear(&Hp);                                /* H~' <- empty */
        Qp.n = 0;                                     /* Q' <- [] */
        for (uint64_t p = 0; p < Q.n; ++p) {
            uint32_t v = Q.a[p].v;
            int32_t k = Q.a[p].k;
            ent_t *e = hm_find(&H, dkey(v, k));
            int32_t j = e->j;
            int64_t b = e->base;
            int64_t i = (int64_t)k + j;               /* i <- k + H~_{v,k} */
            int32_t lv = (int32_t)og_len(&g, v);
            /* three candidates: (k+1, j) insertion, (k-1, j+1) deletion, (k, j+1) mismatch */
            int32_t ck[3] = {k + 1, k - 1, k};
            int32_t cj[3] = {j, j + 1, j + 1};
            int ok[3] = {i < (int64_t)n, j < lv, i < (int64_t)n && j < lv};
            for (int c = 0; c < 3; ++c) {
                if (!ok[c]) continue;
                ent_t *tp = hm_find(&Hp, dkey(v, ck[c]));
                if (!tp) {                            /* H~'_{v,k'} not in H~' */
                    int improves = 1;
                    if (c < 2) {                      /* the mismatch case has no test */
                        ent_t *th = hm_find(&H, dkey(v, ck[c]));
                        improves = !th || th->j < cj[c];
                    }
                    if (improves) {
                        tp = hm_insert(&Hp, dkey(v, ck[c]));
                        if (!tp) { rc = OR_ERR_OOM; goto done; }
                        tp->j = cj[c]; tp->base = b;
                        if (dv_push(&Qp, v, ck[c])) { rc = OR_ERR_OOM; goto done; }
                    }
                } else if (cj[c] > tp->j || (cj[c] == tp->j && b > tp->base)) {
                    tp->j = cj[c]; tp->base = b;      /* max-merge, ties by base */
                }
            }
        }
        for (uint64_t p = 0; p < Qp.n; ++p) {         /* H~_{v,k} <- H~'_{v,k} for (v,k) in Q' */
            ent_t *tp = hm_find(&Hp, dkey(Qp.a[p].v, Qp.a[p].k));
            ent_t *th = hm_find(&H, dkey(Qp.a[p].v, Qp.a[p].k));
            if (!th) {
                th = hm_insert(&H, dkey(Qp.a[p].v, Qp.a[p].k));
                if (!th) { rc = OR_ERR_OOM; goto done; }
                ++inserted;
            }
            th->j = tp->j; th->base = tp->base; th->spill_mark = UINT64_MAX;
        }
        { dvec tq = Q; Q = Qp; Qp = tq; }            /* Q <- Q' */
        if (Q.n == 0) { rc = OR_ERR_EMPTY_FRONTIER; goto done; }

        /* ---- memory bound on H~ (see above) ---- */
        if (evict_lag > 0 && d % evict_every == 0 && !plant_evict_before) {
            rc = evict(&H, plant_evict_oldq ? &Qx : &Q, amax, evict_lag, plant_evict_le, out);
            if (rc) goto done;
            if (plant_evict_oldq) {                 /* the new Q loses what that removed */
                uint64_t m = 0;
                for (uint64_t p = 0; p < Q.n; ++p)
                    if (hm_find(&H, dkey(Q.a[p].v, Q.a[p].k))) Q.a[m++] = Q.a[p];
                Q.n = m;
                if (Q.n == 0) { rc = OR_ERR_EMPTY_FRONTIER; goto done; }
            }
        }
    }
    out->distance = d;
done:
    out->visited = inserted;
    if (rc != OR_OK) out->distance = rc;
    free(H.e); free(Hp.e); free(Q.a); free(Qp.a); free(Qx.a); free(q); og_free(&g);
    return rc;
}

int oracle_gwfa_ends(uint32_t nv, const char *seq, const uint64_t *seq_off,
                     uint64_t na, const uint32_t *asrc, const uint32_t *adst,
                     const char *qs, uint64_t n, uint32_t vs, uint32_t ve,
                     int64_t a_diff, int64_t max_score, int ends, oracle_stats *out) {
    return oracle_gwfa_ex(nv, seq, seq_off, na, asrc, adst, qs, n, vs, ve, a_diff, max_score, ends, 0, 0, out);
}

int oracle_gwfa(uint32_t nv, const char *seq, const uint64_t *seq_off,
                uint64_t na, const uint32_t *asrc, const uint32_t *adst,
                const char *qs, uint64_t n, uint32_t vs, uint32_t ve,
                int64_t a_diff, int64_t max_score, oracle_stats *out) {
    return oracle_gwfa_ends(nv, seq, seq_off, na, asrc, adst, qs, n, vs, ve, a_diff, max_score, 0, out);
}

/* size of oracle_stats, so the python wrapper can check its mirror */
uint64_t oracle_stats_size(void) { return sizeof(oracle_stats); }
