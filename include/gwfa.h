/*
 * gwfa.h -- C ABI of the GB300 graph wavefront alignment library (libgwfa.so).
 *
 * The library aligns DNA queries to a sequence graph G(V, E, sigma) (Def. 1 of
 * "Fast sequence to graph alignment using the graph wavefront algorithm",
 * Zhang, Wu, Aluru & Li): for a query q, a start vertex v_s and an end vertex
 * v_e reachable from v_s, it returns the minimum edit distance between q and
 * the spelled sequence of any walk from v_s to v_e, gaps at both ends penalised
 * (Def. 2, the optimal global sequence-to-graph alignment).  The distance is
 * computed by the graph wavefront algorithm (Alg. 1-3, Eq. 2) and optionally
 * with the lag-based wavefront pruning heuristic (Alg. 4), whose distances are
 * upper bounds.
 *
 * Conventions for every function:
 *   - the return value is a status: GWFA_OK (0) or a negative GWFA_ERR_* code;
 *     gwfa_strerror() gives its text;
 *   - pointers named h_* / plain pointers are host memory, d_* are device
 *     memory of the graph's GPU; the caller keeps ownership of every buffer it
 *     passes and may free or reuse it when the call returns (for *_device calls:
 *     once the work queued on `stream` has completed);
 *   - a `stream` argument is a cudaStream_t passed as void*.  Calls that only
 *     enqueue device work (*_device) use exactly that stream, NULL meaning the
 *     legacy default stream, so they are ordered after whatever produced their
 *     inputs on it; synchronous host-buffer calls use the object's own stream
 *     when it is NULL;
 *   - sequences are ASCII A/C/G/T, either case; anything else is rejected
 *     (GWFA_ERR_INVALID) because sequences are stored 2-bit packed.
 *   - all work runs in CUDA kernels on one GPU; there is no CPU fallback: if the
 *     GPU or the kernels are unavailable the call fails with GWFA_ERR_CUDA.
 */
#ifndef GWFA_H
#define GWFA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define GWFA_OK 0
#define GWFA_PENDING 1              /* serving: request not finished yet */
#define GWFA_ERR_INVALID (-1)       /* bad argument: non-ACGT base, empty label, id out of range */
#define GWFA_ERR_OOM (-2)           /* device or host allocation failed */
#define GWFA_ERR_CUDA (-3)          /* CUDA runtime error / no usable GPU */
#define GWFA_ERR_UNREACHABLE (-4)   /* v_e is not reachable from v_s (Def. 2 requires it) */
#define GWFA_ERR_EMPTY_FRONTIER (-5)/* pruning (Alg. 4) removed every live diagonal */
#define GWFA_ERR_CAPACITY (-6)      /* per-query workspace too small (hash / frontier) */
#define GWFA_ERR_TIMEOUT (-7)       /* a bounded device wait expired */
#define GWFA_ERR_SCORE_LIMIT (-8)   /* distance exceeds opts.max_score */
#define GWFA_ERR_NOT_RUN (-9)       /* query was not processed (batch aborted) */

const char *gwfa_strerror(int status);

/* ---- options and results ------------------------------------------------ */
typedef struct {
    int32_t max_lag;     /* a_diff of Alg. 4 (Sec. 2.5); 0 = exact (no pruning) */
    int32_t traceback;   /* 1: record the alignment walk (Alg. 5-6), with or without
                            pruning; needs 64-bit slabs (engine prune_slabs) and no
                            evict_lag; see gwfa_align_path / gwfa_engine_set_paths */
    int32_t max_score;   /* stop with GWFA_ERR_SCORE_LIMIT once d would exceed it; -1 = no limit */
    int32_t wait_limit;  /* serving: iteration limit of device-side waits; 0 = default */
    int32_t ends;        /* formulation variant (Sec. 2.1), GWFA_FREE_* / GWFA_EXTEND flags;
                            0 = global alignment from the first base of v_s to the last of
                            v_e (Def. 2).  Needs max_lag == 0; the plain path and the
                            batch engine take it, the server and gwfa_align_noalloc
                            refuse it (GWFA_ERR_INVALID) */
    int32_t evict_lag;   /* memory bound on H~ with pruning (max_lag > 0, no traceback): every
                            evict_every scores, right after GwfExpand, the entries outside Q
                            whose anti-diagonal i + W~ lags this score's maximum by evict_lag
                            or more are removed; a removed diagonal may be inserted again
                            (counted again in `visited`).  The distance stays an upper bound;
                            the work counts change and `evicted` reports the removals.  0 = off;
                            batch engine and plain path only */
    int32_t evict_every; /* scores between two evictions; 0 = 64 */
} gwfa_opts;                 /* 28 bytes */

/* Formulation variants: the walk may begin at any position of v_s (its prefix is
 * skipped at no cost), may end at any position of v_e (its suffix skipped), or
 * has no end vertex at all -- the whole query is aligned to a walk that starts
 * at v_s and ends anywhere (v_e is ignored).  A walk may skip a whole end vertex.
 * The reported distance is the minimum over those walks; with traceback the
 * walk runs from v_s to the vertex where the alignment ended. */
#define GWFA_FREE_START 1
#define GWFA_FREE_END 2
#define GWFA_EXTEND 4

/*
 * Per-query result.  Work counters follow Alg. 1-3 exactly and are identical
 * for every execution order (the queue order of Alg. 2-3 does not change them):
 *   n_scores      number of GwfExtend calls (= edit_distance + 1 on success);
 *   cells         sum over scores of |Q| after GwfExtend (diagonals extended);
 *   peak_frontier max over scores of |Q| after GwfExtend;
 *   visited       insertions of diagonals (v, k) into H~: the distinct diagonals ever
 *                 inserted, unless the memory bound removed some that came back;
 *   pruned        diagonals dropped by GwfPrune, summed over scores;
 *   spills        diagonals inserted by the arc loop of GwfExtend.
 */
typedef struct {
    int32_t status;          /* GWFA_OK or GWFA_ERR_* */
    int32_t edit_distance;   /* valid when status == GWFA_OK */
    int32_t is_upper_bound;  /* 1 iff pruning dropped at least one diagonal */
    uint32_t n_scores;
    uint64_t cells;
    uint64_t visited;
    uint32_t peak_frontier;
    uint32_t device_us;      /* device time the CTA spent on this query, microseconds */
    uint64_t pruned;
    uint64_t spills;
    uint64_t evicted;        /* H~ entries removed by the memory bound (opts.evict_lag) */
} gwfa_result;               /* 64 bytes */

/* ---- graph -------------------------------------------------------------- */
typedef struct gwfa_graph gwfa_graph;

/*
 * Upload a sequence graph (Def. 1) to GPU `device` as 2-bit packed labels
 * (16 bases per 32-bit word, each vertex starting on a word boundary) plus a
 * CSR of out-arcs.
 *   n_vertices       |V| (1 .. 2^31)
 *   h_seq, h_seq_off labels concatenated: label v is h_seq[h_seq_off[v] .. h_seq_off[v+1]),
 *                    h_seq_off has n_vertices+1 entries; every label must be non-empty
 *                    (an empty label would create zero-cost cycles) and shorter than 2^30
 *   n_arcs, h_arc_src, h_arc_dst   arcs (u, v) of E; duplicates are merged
 * Errors: GWFA_ERR_INVALID (bad base, empty label, vertex id out of range),
 * GWFA_ERR_OOM, GWFA_ERR_CUDA.  The graph is immutable afterwards and may be
 * shared by any number of engines and threads.
 */
int gwfa_graph_create(uint32_t n_vertices, const char *h_seq, const uint64_t *h_seq_off,
                      uint64_t n_arcs, const uint32_t *h_arc_src, const uint32_t *h_arc_dst,
                      int device, gwfa_graph **out);
int gwfa_graph_destroy(gwfa_graph *g);

typedef struct {
    uint32_t n_vertices;
    uint32_t max_out_degree;
    uint64_t n_arcs;          /* after merging duplicates */
    uint64_t total_bases;
    uint64_t device_bytes;    /* resident footprint of the packed graph */
    int32_t device;
    int32_t has_cycles;       /* 1 if some arc goes to an equal or lower vertex id */
} gwfa_graph_info;
int gwfa_graph_get_info(const gwfa_graph *g, gwfa_graph_info *out);

/* ---- plain path: one query, one kernel launch, synchronous -------------- */
/*
 * Align one query (Alg. 1 with Alg. 2-4) with a single-CTA launch of the same
 * kernel the batched path uses.  Host reachability check first
 * (GWFA_ERR_UNREACHABLE).  Result in *out (host).  Uses a workspace owned by
 * the graph, so concurrent gwfa_align calls on one graph are serialised.
 */
int gwfa_align(const gwfa_graph *g, const char *h_q, uint32_t n, uint32_t v_s, uint32_t v_e,
               const gwfa_opts *opts, gwfa_result *out);

/*
 * gwfa_align with the optimal walk (Alg. 5-6): the vertices of one s->e walk
 * whose spelled sequence is at edit distance out->edit_distance from the query
 * (several optimal walks may exist; this returns one).  h_path[path_cap] gets
 * the first min(path_cap, *path_len) vertex ids; *path_len is the full length.
 * With pruning (opts->max_lag > 0) the walk is the one the pruned wavefront
 * reached the end cell along: the query aligns to its spelled sequence with at
 * most out->edit_distance edits (the upper bound), and with at least the exact
 * distance.
 */
int gwfa_align_path(const gwfa_graph *g, const char *h_q, uint32_t n, uint32_t v_s, uint32_t v_e,
                    const gwfa_opts *opts, gwfa_result *out, uint32_t *h_path, uint32_t path_cap,
                    uint32_t *path_len);

/* ---- batched path: persistent kernel with a device work queue ----------- */
typedef struct gwfa_engine gwfa_engine;

/*
 * Engine = device workspace for batched alignment.  Each CTA of the persistent
 * kernel owns one slab (per-query hash of diagonal tiles + frontier lists) and
 * pulls query ids from an atomic queue; a query whose slab overflows is put on
 * a retry list and re-run by the next tier (fewer CTAs, larger slabs) in the
 * same stream, without a host round trip.
 *   tiers[t].ctas  CTAs of tier t
 *   tiers[t].log2_tiles  slab capacity in 8-diagonal tiles (log2)
 *   tiers[t].threads     threads per CTA of tier t (0 = `threads`)
 *   huge, wide     two extra classes of CTAs (usually with larger slabs) that run
 *                  concurrently with tier 0 on the first n_huge, then the next
 *                  n_wide queries of the schedule (gwfa_schedule), so the heaviest
 *                  queries start at once on slabs that fit them instead of forming a
 *                  tail of overflow re-runs; their overflows go to the retry tiers
 *   threads        threads per CTA (multiple of 32, 32..1024; above 512 a CTA
 *                  takes half an SM: for the few heaviest queries, e.g. the huge
 *                  class, whose own latency bounds a batch); 0 = 128
 *   max_queries, max_bases  sizes of the engine's staging buffers for the
 *                  host-buffer entry point (grown on demand)
 */
#define GWFA_MAX_TIERS 4
typedef struct {
    uint32_t ctas;
    uint32_t log2_tiles;
    uint32_t threads;         /* threads per CTA of this tier; 0 = the config's `threads` */
    uint32_t reserved;
} gwfa_tier;

typedef struct {
    uint32_t n_tiers;
    gwfa_tier tiers[GWFA_MAX_TIERS];
    gwfa_tier wide;           /* CTAs for heavy queries, run beside tier 0; ctas 0 = none */
    gwfa_tier huge;           /* CTAs with very large slabs for the heaviest, beside tier 0 */
    uint32_t threads;
    uint32_t prune_slabs;     /* 1: size slabs for pruning mode (64-bit offsets) */
    uint64_t max_queries;
    uint64_t max_bases;
} gwfa_engine_config;

/* Placement of a batch: queue positions [0, n_huge) run on the huge class,
 * [n_huge, n_huge + n_wide) on the wide class, the rest on tier 0. */
typedef struct {
    uint32_t n_huge;
    uint32_t n_wide;
} gwfa_schedule;

/* fills a default configuration for this GPU (3 tiers, 512 threads, no classes) */
int gwfa_engine_default_config(const gwfa_graph *g, int prune, gwfa_engine_config *cfg);
int gwfa_engine_create(const gwfa_graph *g, const gwfa_engine_config *cfg, gwfa_engine **out);
int gwfa_engine_destroy(gwfa_engine *e);
/* bytes of device memory held by the engine */
uint64_t gwfa_engine_device_bytes(const gwfa_engine *e);

/*
 * Host-buffer batch (end to end).  Queries concatenated in h_q (ASCII) with
 * h_q_off[n_queries+1] byte offsets, per-query start/end vertices in
 * h_v_s / h_v_e.  h_order (may be NULL = input order) is the order in which the
 * work queue hands queries to CTAs (a permutation of 0..n_queries-1), placed by
 * `sched` (NULL = all on tier 0).  The call
 * copies the inputs to the device, packs them (kernel), runs the tiers, copies
 * the n_queries results to h_out and returns when they are there.  Per-query
 * errors are in h_out[i].status; the return value is the first fatal error.
 * For pinned host buffers the copies are asynchronous DMA.
 */
int gwfa_align_batch(gwfa_engine *e, uint32_t n_queries, const char *h_q, const uint64_t *h_q_off,
                     const uint32_t *h_v_s, const uint32_t *h_v_e, const uint32_t *h_order,
                     const gwfa_schedule *sched, const gwfa_opts *opts, gwfa_result *h_out,
                     void *stream);

/*
 * Device-resident packing of queries (the step gwfa_align_batch runs after its
 * copy): d_q / d_q_off as above but in device memory; writes 2-bit words to
 * d_words with query i starting at word (d_q_off[i] >> 4) + i, so d_words needs
 * (q_off[n] >> 4) + n_queries + 2 words.  Queries with a non-ACGT base get
 * status GWFA_ERR_INVALID in d_status (int32[n_queries]) and 0 otherwise.
 */
int gwfa_pack_queries_device(uint32_t n_queries, const char *d_q, const uint64_t *d_q_off,
                             uint32_t *d_words, int32_t *d_status, void *stream);

/*
 * Device-resident batch (inputs already in HBM): d_words / d_q_off as written
 * by gwfa_pack_queries_device (d_status may be NULL, else queries with a
 * nonzero status are skipped and keep it), d_v_s / d_v_e start/end vertices,
 * d_order the queue order (NULL = 0..n-1) placed by `sched` (NULL = all on
 * tier 0; host memory), results into d_out[n_queries].
 * Asynchronous on `stream`; no host synchronisation inside.
 */
int gwfa_align_batch_device(gwfa_engine *e, uint32_t n_queries, const uint32_t *d_words,
                            const uint64_t *d_q_off, const uint32_t *d_v_s, const uint32_t *d_v_e,
                            const uint32_t *d_order, const gwfa_schedule *sched,
                            const int32_t *d_status, const gwfa_opts *opts, gwfa_result *d_out,
                            void *stream);

/*
 * Allocation-free batch alignment (no counterpart in the paper: it exists for
 * callers that cannot let a library allocate device memory -- code running
 * inside a custom device-memory allocator, where calling back into allocation
 * can deadlock or recurse; processes whose device memory another framework has
 * reserved up front; loops that cannot afford cudaMalloc's implicit device-wide
 * synchronisation).  Same kernel and same results as gwfa_align_batch_device,
 * but its scratch is one fixed 32 MiB device array inside the library (present
 * on every GPU that loads it, until the process exits), carved into
 * floor((32 MiB - 256 B) / slab) CTA slabs of 2^log2_tiles hash tiles each
 * (log2_tiles 0 = 15: five CTAs in exact mode, two with pruning).  There is
 * no overflow tier: a query needing more than 3/4 of its slab gets status
 * GWFA_ERR_CAPACITY.  log2_tiles outside [8, 24] (other than 0) is
 * GWFA_ERR_INVALID; a valid log2_tiles whose slab does not fit the array is
 * rejected with GWFA_ERR_CAPACITY, both before any GPU work.  Inputs and outputs
 * are the caller's device buffers, laid out as for gwfa_align_batch_device
 * (d_words from gwfa_pack_queries_device); d_status may be NULL, else it is the
 * status array that packing wrote, and a query with a nonzero status (a base
 * other than A/C/G/T) is not aligned and keeps that status in d_out, as in
 * gwfa_align_batch_device.  With d_status NULL such a query is aligned with its
 * bad bases read as A.  The call only enqueues work on `stream` (NULL = the
 * legacy default stream) and calls no allocation routine.
 * The first call on a device looks up the array's device address (once per
 * device, and again if a device reset replaced the context); make that first
 * call before any stream capture.  Every call shares the array and resets it
 * first, so calls whose GPU work overlaps race on it: the caller must serialise
 * them (one stream, or its own ordering).
 */
int gwfa_align_noalloc(const gwfa_graph *g, uint32_t n_queries, const uint32_t *d_words,
                       const uint64_t *d_q_off, const uint32_t *d_v_s, const uint32_t *d_v_e,
                       const int32_t *d_status, uint32_t log2_tiles, const gwfa_opts *opts,
                       gwfa_result *d_out, void *stream);

/* Walk output of later batch calls with opts.traceback = 1: query i writes its
 * walk to d_paths[i * path_cap ...] (at most path_cap ids) and its full length to
 * d_path_len[i]; both device buffers are the caller's (NULL / 0 = off). */
int gwfa_engine_set_paths(gwfa_engine *e, uint32_t *d_paths, uint32_t path_cap, uint32_t *d_path_len);

/* number of kernel launches the last batch call on this engine queued */
uint32_t gwfa_engine_last_launches(const gwfa_engine *e);

/*
 * Per-query statistics of later batch calls on this engine (NULL = off): the
 * kernels write 8 uint64 per query id into d_stats (device memory of
 * n_queries * 8 words, owned by the caller, valid until replaced): time spent in
 * GwfExtend and in GwfExpand (ns, measured by the CTA), extension rounds,
 * tiles extended, tiles expanded, largest expanded-tile count of a score, tiles
 * claimed in the hash, and the number of scores.  These are the wavefront sizes
 * the learned cost model trains on.
 */
int gwfa_engine_set_stats(gwfa_engine *e, uint64_t *d_stats);

/* tier-0 overflows of the last batch call, per tier boundary (synchronises the engine's
 * last stream): out[t] = queries that tier t handed to tier t+1 (t < GWFA_MAX_TIERS - 1) */
int gwfa_engine_last_retries(gwfa_engine *e, uint32_t *out);

/* ---- base-level alignment along the walk -------------------------------- */
/*
 * Gwfa returns a distance and (Alg. 5-6) a vertex walk, not a base-level
 * alignment; the paper's discussion (Sec. 4) obtains one by aligning the query
 * to the sequence the walk spells with a pairwise method.  This step does that on
 * the device: for each query it spells sigma(w) (2-bit packed) and runs a
 * pairwise edit-distance wavefront alignment (unit costs) bounded by the query's
 * reported distance, then walks the stored wavefronts back to a CIGAR.  The ends
 * follow the batch's formulation (`ends`, GWFA_FREE_* / GWFA_EXTEND): the query is
 * always aligned whole; the walk's first vertex may be entered past its start
 * under GWFA_FREE_START, its last vertex left before its end under GWFA_FREE_END
 * or GWFA_EXTEND; [walk_begin, walk_end) is the aligned part of sigma(w).  When w
 * is optimal the CIGAR has exactly edit_distance edits.
 *
 * CIGAR operations are uint32 (length << 4 | op) with the BAM op codes below,
 * query = the read, walk = the reference: '=' a run of equal bases, 'X' one
 * substituted base, 'I' a query base absent from the walk, 'D' a walk base absent
 * from the query.  Adjacent operations of one kind are merged.
 */
#define GWFA_CIGAR_INS 1
#define GWFA_CIGAR_DEL 2
#define GWFA_CIGAR_EQ 7
#define GWFA_CIGAR_DIFF 8
typedef struct gwfa_cigar gwfa_cigar;
typedef struct {
    int32_t status;       /* GWFA_OK; GWFA_ERR_NOT_RUN (the query's alignment did not
                             succeed); GWFA_ERR_CAPACITY (walk truncated at path_cap,
                             workspace too small, or more than cigar_cap operations:
                             n_ops still tells how many); GWFA_ERR_SCORE_LIMIT (the walk
                             is farther than edit_distance from the query) */
    int32_t cost;         /* edits of the CIGAR */
    uint32_t n_ops;       /* CIGAR operations */
    uint32_t walk_len;    /* bases spelled by the walk */
    uint32_t walk_begin;  /* first aligned base of sigma(w) (0 unless GWFA_FREE_START) */
    uint32_t walk_end;    /* one past the last aligned base (walk_len unless a free end) */
} gwfa_cigar_result;      /* 24 bytes */

/*
 * ctas: persistent CTAs (0 = 2 per SM); workspace_bytes: device scratch per CTA
 * (0 = 32 MiB).  Only every c-th pairwise wavefront is kept, c = ceil(sqrt(d + 1)),
 * and the others are recomputed segment by segment during the backtrace, so a
 * query needs 4 * (|sigma(w)| / 16 + 2) + 4 * (d / c + c + 2) * (2 d + L + 1)
 * bytes (the first term rounded up to 16; L = |first vertex| under GWFA_FREE_START,
 * else 0): the default holds distances up to ~1.7 x 10^4 on walks of 100 kb.  The
 * workspace is allocated here; gwfa_cigar_device allocates nothing.
 */
int gwfa_cigar_create(const gwfa_graph *g, uint32_t ctas, uint64_t workspace_bytes, gwfa_cigar **out);
int gwfa_cigar_destroy(gwfa_cigar *c);
/*
 * Asynchronous on `stream` (NULL = legacy default stream), device pointers:
 *   d_words, d_q_off  the packed batch (as for gwfa_align_batch_device)
 *   d_res             the batch's results (status, edit_distance are read)
 *   d_paths, path_cap, d_path_len   the walks written by a traceback batch
 *                     (gwfa_engine_set_paths)
 *   d_cigar           n_queries * cigar_cap operations; query i writes from
 *                     d_cigar[i * cigar_cap]
 *   d_out             n_queries results
 *   ends              the formulation flags the batch was aligned with
 * Calls on one gwfa_cigar share its workspace: order them on one stream.
 */
int gwfa_cigar_device(gwfa_cigar *c, uint32_t n_queries, const uint32_t *d_words,
                      const uint64_t *d_q_off, const gwfa_result *d_res, const uint32_t *d_paths,
                      uint32_t path_cap, const uint32_t *d_path_len, uint32_t *d_cigar,
                      uint32_t cigar_cap, int32_t ends, gwfa_cigar_result *d_out, void *stream);

/* ---- learned cost model (scheduling only; never changes a result) -------- */
/*
 * A 6 -> 32 -> 32 -> 4 MLP (ReLU; FP16 weights and activations, FP32
 * accumulation and FP32 master weights) predicts per query, in log1p units:
 *   0 the edit distance (scores of Alg. 1), 1 the peak |Q| after GwfExtend,
 *   2 the diagonals that enter H~ (hash memory), 3 the cells (total work).
 * These are the work counters of gwfa_result; the model is trained on them by
 * the library's own forward/backward/Adam kernels.  Parameters (fp32, 1412):
 * W1[32][6], b1[32], W2[32][32], b2[32], W3[4][32], b3[4].
 * Raw features (computed on the device, z-scored inside the model with the
 * normalisation set by gwfa_model_set_normalization):
 *   0 log1p(|q|); 1 fraction of 64 evenly spaced query 16-mers that occur in no
 *   vertex label; 2 log1p(vertices with id between v_s and v_e); 3 log1p(arcs
 *   leaving them); 4 vertices with out-degree > 1 among them per kb of query;
 *   5 log1p(arcs from them to an equal or lower id).
 */
#define GWFA_MODEL_FEATURES 6
#define GWFA_MODEL_TARGETS 4
#define GWFA_MODEL_PARAMS 1412
typedef struct gwfa_model gwfa_model;

/* builds the graph's feature tables (sorted 16-mers of the labels, prefix counts)
 * on the graph's device and initialises the weights from `seed` */
int gwfa_model_create(const gwfa_graph *g, uint64_t seed, gwfa_model **out);
int gwfa_model_destroy(gwfa_model *m);
int gwfa_model_set_params(gwfa_model *m, const float *h_params, uint32_t n_params);
int gwfa_model_get_params(const gwfa_model *m, float *h_params, uint32_t n_params);
/* feature means/stds (GWFA_MODEL_FEATURES each) and target means/stds (GWFA_MODEL_TARGETS) */
int gwfa_model_set_normalization(gwfa_model *m, const float *h_fmean, const float *h_fstd,
                                 const float *h_tmean, const float *h_tstd);
/* write the weights and the normalisation to a file at `path` / read them back
 * (the parameter and normalisation shapes are checked); GWFA_ERR_INVALID for a file
 * that cannot be opened, written or parsed.  Both synchronise the model's device. */
int gwfa_model_save(const gwfa_model *m, const char *path);
int gwfa_model_load(gwfa_model *m, const char *path);
/* raw features of n packed queries (layout of gwfa_pack_queries_device) into d_feat[n][6] */
int gwfa_model_features_device(gwfa_model *m, uint32_t n, const uint32_t *d_words,
                               const uint64_t *d_q_off, const uint32_t *d_v_s, const uint32_t *d_v_e,
                               float *d_feat, void *stream);
/* predictions d_pred[n][4] (log1p units) from raw features */
int gwfa_model_predict_device(gwfa_model *m, uint32_t n, const float *d_feat, float *d_pred,
                              void *stream);
/* gradient of the mean squared error over all n samples (targets d_target[n][4] in
 * log1p units, compared after normalisation) at the current weights, into
 * h_grad[1412]; *h_loss = the loss.  Synchronous. */
int gwfa_model_gradient_device(gwfa_model *m, uint32_t n, const float *d_feat, const float *d_target,
                               float *h_grad, float *h_loss, void *stream);
/* `steps` Adam steps (lr, beta 0.9 / 0.999) on minibatches of `batch` samples drawn
 * as slices of seeded permutations; h_losses[steps] (may be NULL) gets each step's
 * minibatch loss.  Synchronous. */
int gwfa_model_train_device(gwfa_model *m, uint32_t n, const float *d_feat, const float *d_target,
                            uint32_t steps, uint32_t batch, float lr, uint64_t seed, float *h_losses,
                            void *stream);

/* the same prediction for one ASCII query, evaluated on the host in fp32 with the
 * current weights (used for admission control in serving) */
int gwfa_model_predict_host(const gwfa_model *m, const char *h_q, uint32_t n, uint32_t v_s,
                            uint32_t v_e, float *h_pred);

/*
 * Batch plan from predicted costs (host, no GPU): the queries whose predicted hash
 * tiles exceed `wide_tiles` (0 = no huge class) come first (out->n_huge), then
 * those exceeding `tier0_tiles` (out->n_wide), then the rest, each group by
 * decreasing predicted cells (longest processing time first), so the heavy
 * queries start at once on slabs that fit them instead of overflowing tier 0 and
 * being re-run.
 *   h_pred  n x 4 predictions (log1p units, as from gwfa_model_predict_device)
 */
int gwfa_plan_schedule(uint32_t n, const float *h_pred, uint64_t tier0_tiles, uint64_t wide_tiles,
                       uint32_t *h_order, gwfa_schedule *out);

/* ---- serving: continuous batching over a resident graph ----------------- */
/*
 * A persistent kernel keeps the graph resident and takes requests as its CTAs
 * free up; requests submitted while others are on the GPU start without waiting
 * for a batch boundary.  Requests and results pass through pinned host memory
 * mapped into the device.  Two request classes: CTAs with small hash slabs
 * (ctas_small, 2^log2_small tiles) and CTAs with large ones (ctas_big,
 * 2^log2_big); a request enters the class its predicted hash memory fits (the
 * attached cost model, else length > big_length), and a request that overflows
 * a small slab is re-queued into the large class automatically.  Large-slab CTAs
 * also take small requests whenever no large one waits.  The default configuration
 * (gwfa_server_default_config) puts 2^17-tile slabs on 4 x SMs - SMs / 2 CTAs and
 * 2^21-tile slabs on SMs / 2 CTAs of 512 threads (about 41 GB of device memory in
 * exact mode, 2.3 times that with pruning).  The kernel's
 * CTAs leave together once all of them have been idle for idle_us (and in any
 * case after 16 x idle_us idle; every device wait is bounded), and the next
 * submit or poll starts it again.  Results are identical to gwfa_align.
 * Thread-safe (one internal lock).
 */
typedef struct gwfa_server gwfa_server;
typedef struct {
    uint32_t threads;          /* per CTA */
    uint32_t ctas_small, log2_small;
    uint32_t ctas_big, log2_big;
    uint32_t ring_slots;       /* requests in flight per class */
    uint32_t max_query_len;    /* longer requests are rejected (GWFA_ERR_INVALID) */
    uint32_t idle_us;          /* idle time after which the kernel's CTAs leave */
    uint32_t big_length;       /* without a cost model: class 1 iff |q| > big_length */
} gwfa_server_config;

typedef struct {
    uint64_t submitted, completed, requeued, launches, in_flight, device_bytes;
} gwfa_server_stats;

int gwfa_server_default_config(const gwfa_graph *g, gwfa_server_config *cfg);
/* `model` (may be NULL) must outlive the server */
int gwfa_server_create(const gwfa_graph *g, const gwfa_server_config *cfg, const gwfa_opts *opts,
                       const gwfa_model *model, gwfa_server **out);
/* GWFA_OK with *ticket set, GWFA_PENDING when the class's ring is full (retry later),
 * GWFA_ERR_INVALID for a bad query */
int gwfa_submit(gwfa_server *s, const char *h_q, uint32_t n, uint32_t v_s, uint32_t v_e,
                uint64_t *ticket);
/* GWFA_OK with *out filled (once per ticket), or GWFA_PENDING */
int gwfa_poll(gwfa_server *s, uint64_t ticket, gwfa_result *out);
/* gwfa_poll over tickets[i] whose done_flags[i] is 0: finished ones get out[i] and
 * done_flags[i] = 1; *n_done = how many finished in this call */
int gwfa_poll_many(gwfa_server *s, uint32_t n, const uint64_t *tickets, gwfa_result *out,
                   uint8_t *done_flags, uint32_t *n_done);
/* polls until done or timeout_ms (GWFA_ERR_TIMEOUT) */
int gwfa_wait(gwfa_server *s, uint64_t ticket, uint32_t timeout_ms, gwfa_result *out);
int gwfa_server_get_stats(gwfa_server *s, gwfa_server_stats *out);
/* stops the kernel (requests on the GPU finish first) and frees everything */
int gwfa_server_destroy(gwfa_server *s);

/* ---- measurement -------------------------------------------------------- */
/*
 * Integer-pipe ceiling of `device` (used to report the alignment kernels against
 * their roofline; the paper has no counterpart -- its complexity analysis, Sec. 2.4,
 * bounds the work, not the machine).  Runs a kernel of blocks_per_sm (0 = 2)
 * 1024-thread CTAs per SM in which every thread issues `iters` x 64 independent
 * 3-input logic operations (lop3, ALU pipe, no memory traffic), four times on a
 * private stream; *ms_out = the fastest of the last three runs (CUDA events) and
 * *warp_insts_out = the lop3 warp instructions one run issues.  Their ratio is the
 * ALU-pipe warp-instruction rate of the whole GPU.  Synchronous; allocates nothing
 * but a stream and two events.  GWFA_ERR_INVALID for NULL outputs or iters = 0.
 */
int gwfa_measure_int_peak(int device, uint32_t blocks_per_sm, uint32_t iters, float *ms_out,
                          uint64_t *warp_insts_out);

#ifdef __cplusplus
}
#endif
#endif /* GWFA_H */
