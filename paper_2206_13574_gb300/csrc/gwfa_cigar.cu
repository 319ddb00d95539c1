// gwfa_cigar.cu -- base-level alignment of each query to the sequence its walk spells.
//
// Gwfa (Alg. 1-6) yields the edit distance and one optimal vertex walk w.  The
// paper's discussion (Sec. 4) gets the base-level alignment by aligning the query
// to sigma(w) with a pairwise method; here that is an edit-distance wavefront
// alignment on the device, one persistent CTA per query at a time:
//
//   1. spell sigma(w) into the CTA's workspace, 2-bit packed like the graph labels
//      (a block-wide prefix sum of the label lengths gives each vertex's position);
//   2. for s = 0, 1, ... compute the furthest point of every diagonal k = j - i
//      (i in the query, j in the walk) at score s from score s - 1 (substitution
//      i+1, j+1; query base skipped i+1; walk base skipped j+1) and extend it along
//      equal bases 16 at a time (XOR of packed windows, first set bit).  Score 0
//      starts at (0, 0), or at every (0, j) of the first vertex when the walk may
//      start inside it (L = its length, else L = 0), so score s spans diagonals
//      -s .. L + s.  Only every c-th wavefront is kept (a checkpoint), with
//      c = ceil(sqrt(d + 1));
//   3. once an end point is on a wavefront -- (n, m), or (n, j) for any j in the
//      last vertex when the walk may end inside it -- the wavefronts are walked
//      back one segment of c scores at a time, last segment first: the CTA
//      recomputes the segment's wavefronts from its checkpoint (each is a
//      deterministic function of the one before, so they are the forward pass's),
//      then one thread steps back through them, each step re-deriving which
//      predecessor gave the point's starting offset and emitting the run of equal
//      bases and one edit.
//
// The score loop is bounded by the query's Gwfa distance d: when w is optimal,
// the pairwise distance of q and sigma(w) (with the same free ends) is d (an
// alignment of q to a walk is an alignment to its spelled sequence and back).
// Rows are 2d + L + 1 offsets wide; ceil(d / c) + 1 checkpoints plus c segment
// rows -- about 2 sqrt(d) rows instead of the d + 1 of keeping every wavefront --
// so distances of 10^4 on 100 kb walks take ~16 MB, for twice the forward work.
#include <cuda_runtime.h>
#include <stdint.h>

#include <new>

#include "gwfa_internal.cuh"

struct gwfa_cigar {
    const gwfa_graph *g = nullptr;
    uint32_t ctas = 0;
    uint64_t ws_bytes = 0;    // per CTA
    uint8_t *ws = nullptr;    // ctas * ws_bytes
    uint32_t *head = nullptr; // work-queue counter
};

namespace {

constexpr int kThreads = 256;

struct CigarArgs {
    gwfa::DevGraph g;
    const uint32_t *qwords;
    const uint64_t *q_off;
    const gwfa_result *res;
    const uint32_t *paths;
    uint32_t path_cap;
    const uint32_t *path_len;
    uint32_t *cigar;
    uint32_t cigar_cap;
    gwfa_cigar_result *out;
    int ends;
    uint8_t *ws;
    uint64_t ws_bytes;
    uint32_t n;
    uint32_t *head;
};

// 16 bases from base position p of a packed stream (base t of a word in bits
// 2t..2t+1); the query words are read-only here, the walk words are written by
// this CTA, so they are read from L2.
__device__ __forceinline__ uint32_t q16(const uint32_t *w, uint64_t p) {
    const uint64_t i = p >> 4;
    return __funnelshift_r(__ldg(w + i), __ldg(w + i + 1), (uint32_t)(p & 15) * 2);
}
__device__ __forceinline__ uint32_t t16(const uint32_t *w, uint64_t p) {
    const uint64_t i = p >> 4;
    return __funnelshift_r(__ldcg(w + i), __ldcg(w + i + 1), (uint32_t)(p & 15) * 2);
}

// length of the run of equal bases q[i..] / t[j..], at most maxl
__device__ int run_length(const uint32_t *qw, int i, const uint32_t *tw, int j, int maxl) {
    int l = 0;
    while (l < maxl) {
        const uint32_t x = q16(qw, (uint64_t)(i + l)) ^ t16(tw, (uint64_t)(j + l));
        if (x) {
            l += (__ffs(x) - 1) >> 1;
            break;
        }
        l += 16;
    }
    return min(l, maxl);
}

// The three predecessors of diagonal k at score s (prev = wavefront s - 1, indexed
// by diagonal, spanning lo .. hi): the query offset each would start k at, or -1
// where the move is impossible (unreached predecessor, or it would leave the
// n x m rectangle).
struct Pred {
    int sub, ins, del;
};
__device__ __forceinline__ Pred predecessors(const int *prev, int lo, int hi, int k, int n, int m) {
    Pred p{-1, -1, -1};
    if (k >= lo && k <= hi) {
        const int v = __ldcg(prev + k);
        if (v >= 0 && v < n && v + k < m) p.sub = v + 1;        // (v, v+k) -> (v+1, v+k+1)
    }
    if (k + 1 >= lo && k + 1 <= hi) {
        const int v = __ldcg(prev + k + 1);
        if (v >= 0 && v < n) p.ins = v + 1;                     // (v, v+k+1) -> (v+1, v+k+1)
    }
    if (k - 1 >= lo && k - 1 <= hi) {
        const int v = __ldcg(prev + k - 1);
        if (v >= 0 && v + k - 1 < m) p.del = v;                 // (v, v+k-1) -> (v, v+k)
    }
    return p;
}

// Stored wavefronts: fixed-width rows of W = 2d + L + 1 offsets, diagonal k of a
// row at index k + d (score s only fills -s .. L + s).  Rows [0, n_ck) are the
// checkpoints (score r * c in row r), rows n_ck .. n_ck + c - 1 the segment being
// recomputed (score b + t in row n_ck + t; the forward pass uses two of them in
// turn).
struct Rows {
    int *base;
    int64_t width;
    int d, c, n_ck;
    __device__ int *row(int r) const { return base + (int64_t)r * width + d; }
    __device__ int *checkpoint(int s) const { return row(s / c); }
    __device__ int *segment(int t) const { return row(n_ck + t); }
};

// Wavefront s (diagonals -s .. L + s) from wavefront s - 1 (NULL for s = 0); true if
// it reaches an end point, whose smallest diagonal goes to *s_hitk (shared memory;
// NULL when recomputing a wavefront already known to reach none).
__device__ bool wavefront_step(int s, const int *prev, int *cur, int L, int n, int m, const uint32_t *qw,
                               const uint32_t *tw, bool free_end, int l_last, int k_end, int *s_hitk) {
    bool hit = false;
    for (int k = -s + (int)threadIdx.x; k <= L + s; k += blockDim.x) {
        int c = -1;
        if (s == 0) {
            c = k >= 0 ? 0 : -1;   // (0, k): the walk entered k bases into its first vertex
        } else {
            const Pred p = predecessors(prev, -(s - 1), L + s - 1, k, n, m);
            c = max(p.sub, max(p.ins, p.del));
        }
        int i = -1;
        if (c >= 0 && c <= n && c + k >= 0 && c + k <= m)
            i = c + run_length(qw, c, tw, c + k, min(n - c, m - c - k));
        __stcg(cur + k, i);
        if (s_hitk && i == n && (free_end ? n + k >= m - l_last && n + k <= m : k == k_end)) {
            hit = true;
            atomicMin(s_hitk, k);   // several end points: keep the smallest diagonal
        }
    }
    return hit;
}

struct Runs {
    uint32_t *ops;
    uint32_t cap, n, op, len;
    __device__ void emit(uint32_t o, uint32_t l) {
        if (!l) return;
        if (len && o == op) {
            len += l;
            return;
        }
        flush();
        op = o;
        len = l;
    }
    __device__ void flush() {
        if (len) {
            if (n < cap) ops[n] = (len << 4) | op;
            ++n;
        }
        len = 0;
    }
};

__device__ void align_walk(const CigarArgs &A, uint32_t qid, uint32_t *tw, unsigned long long &s_sum,
                           uint32_t *s_warp, uint32_t &s_base, int &s_hitk) {
    const int tid = threadIdx.x;
    const gwfa_result r = A.res[qid];
    const uint32_t plen = A.path_len[qid];
    gwfa_cigar_result o = {GWFA_OK, 0, 0, 0, 0, 0};
    if (r.status != GWFA_OK || plen == 0) o.status = GWFA_ERR_NOT_RUN;
    else if (plen > A.path_cap) o.status = GWFA_ERR_CAPACITY;
    if (o.status) {   // uniform: every thread read the same words
        if (tid == 0) A.out[qid] = o;
        return;
    }
    const uint32_t *walk = A.paths + (uint64_t)qid * A.path_cap;

    // |sigma(w)|
    if (tid == 0) s_sum = 0;
    __syncthreads();
    unsigned long long part = 0;
    for (uint32_t i = tid; i < plen; i += blockDim.x) {
        const uint32_t v = __ldg(walk + i);
        part += v < A.g.nv ? __ldg(&A.g.vinfo[v]).y : (1ull << 40);   // a bad id fails the size test
    }
    atomicAdd(&s_sum, part);
    __syncthreads();
    const unsigned long long m64 = s_sum;
    const int n = (int)(A.q_off[qid + 1] - A.q_off[qid]);
    const int d = r.edit_distance;
    // free ends: lengths of the first and last vertices (0 = the end is fixed)
    const uint32_t v_first = __ldg(walk), v_last = __ldg(walk + plen - 1);
    const int L = (A.ends & GWFA_FREE_START) && v_first < A.g.nv ? (int)__ldg(&A.g.vinfo[v_first]).y : 0;
    const bool free_end = (A.ends & (GWFA_FREE_END | GWFA_EXTEND)) != 0;
    const int l_last = free_end && v_last < A.g.nv ? (int)__ldg(&A.g.vinfo[v_last]).y : 0;
    const uint64_t t_words = (m64 >> 4) + 2;
    const uint64_t wf_off = (t_words * 4 + 15) & ~15ull;
    int seg = 1;   // c = ceil(sqrt(d + 1))
    while ((int64_t)seg * seg < (int64_t)d + 1) ++seg;
    const int n_ck = d / seg + 1;
    const int64_t width = 2 * (int64_t)d + L + 1;
    const uint64_t need = wf_off + (uint64_t)(n_ck + seg + 1) * (uint64_t)width * 4;
    o.walk_len = (uint32_t)min(m64, 0xFFFFFFFFull);
    if (m64 > 0x3FFFFFFFull || d < 0 || need > A.ws_bytes) {
        if (tid == 0) {
            o.status = GWFA_ERR_CAPACITY;
            A.out[qid] = o;
        }
        return;
    }
    const int m = (int)m64;

    // 1. spell sigma(w): zero the words, then OR every label in at its position
    for (uint64_t w = tid; w < t_words; w += blockDim.x) __stcg(tw + w, 0u);
    if (tid == 0) s_base = 0;
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5;
    for (uint32_t c0 = 0; c0 < plen; c0 += blockDim.x) {
        const uint32_t i = c0 + tid;
        uint4 vi = make_uint4(0u, 0u, 0u, 0u);
        if (i < plen) vi = __ldg(&A.g.vinfo[__ldg(walk + i)]);
        uint32_t x = vi.y;   // inclusive scan of the lengths in the warp
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        uint32_t before = s_base;
        for (int w = 0; w < warp; ++w) before += s_warp[w];
        const uint32_t pos = before + x - vi.y;
        const uint32_t *src = A.g.words + vi.x;
        for (uint32_t b = 0; b < vi.y; b += 16) {
            uint32_t w = __ldg(src + (b >> 4));
            const uint32_t nb = min(16u, vi.y - b);
            if (nb < 16) w &= (1u << (2 * nb)) - 1u;
            const uint32_t p = pos + b, sh = (p & 15) * 2;
            atomicOr(tw + (p >> 4), w << sh);
            if (sh) atomicOr(tw + (p >> 4) + 1, w >> (32 - sh));
        }
        __syncthreads();
        if (tid == (int)blockDim.x - 1) s_base = pos + vi.y;
        __syncthreads();
    }

    // 2. wavefronts, score by score, until an end point is reached; checkpoints only
    const Rows R{(int *)((uint8_t *)tw + wf_off), width, d, seg, n_ck};
    const uint32_t *qw = A.qwords + (A.q_off[qid] >> 4) + qid;
    const int k_end = m - n;
    if (tid == 0) s_hitk = 0x7FFFFFFF;
    __syncthreads();
    int found = -1;
    const int *prev = nullptr;
    for (int s = 0; s <= d; ++s) {
        int *cur = s % seg == 0 ? R.checkpoint(s) : R.segment(s & 1);
        const bool hit = wavefront_step(s, prev, cur, L, n, m, qw, tw, free_end, l_last, k_end, &s_hitk);
        if (__syncthreads_or(hit)) {
            found = s;
            break;
        }
        prev = cur;
    }
    if (found < 0) {
        if (tid == 0) {
            o.status = GWFA_ERR_SCORE_LIMIT;
            A.out[qid] = o;
        }
        return;
    }

    // 3. walk back from the end point to score 0, one segment of c scores at a
    // time, last first: wavefronts b + 1 .. b + c - 1 are recomputed from the
    // checkpoint b, then the steps of scores b + c .. b + 1 read them
    __shared__ int s_i, s_k;
    __shared__ uint32_t s_nops, s_op, s_len;
    if (tid == 0) {
        s_i = n;
        s_k = s_hitk;
        s_nops = s_op = s_len = 0;
        o.walk_end = (uint32_t)(n + s_hitk);
    }
    for (int b = ((found - 1) / seg) * seg; found > 0 && b >= 0; b -= seg) {
        const int top = min(b + seg, found);   // steps s = top .. b + 1 read rows top - 1 .. b
        for (int r = b + 1; r <= top - 1; ++r) {
            const int *pr = r - 1 == b ? R.checkpoint(b) : R.segment(r - 1 - b);
            wavefront_step(r, pr, R.segment(r - b), L, n, m, qw, tw, false, 0, 0, nullptr);
            __syncthreads();
        }
        if (tid == 0) {
            Runs Rn{A.cigar + (uint64_t)qid * A.cigar_cap, A.cigar_cap, s_nops, s_op, s_len};
            int i = s_i, k = s_k;
            for (int s = top; s > b; --s) {
                const int *pv = s - 1 == b ? R.checkpoint(b) : R.segment(s - 1 - b);
                const Pred p = predecessors(pv, -(s - 1), L + s - 1, k, n, m);
                const int c = max(p.sub, max(p.ins, p.del));
                Rn.emit(GWFA_CIGAR_EQ, (uint32_t)(i - c));
                if (p.sub == c) {
                    Rn.emit(GWFA_CIGAR_DIFF, 1u);
                    i = c - 1;
                } else if (p.ins == c) {
                    Rn.emit(GWFA_CIGAR_INS, 1u);
                    i = c - 1;
                    k = k + 1;
                } else {
                    Rn.emit(GWFA_CIGAR_DEL, 1u);
                    i = c;
                    k = k - 1;
                }
            }
            s_i = i;
            s_k = k;
            s_nops = Rn.n;
            s_op = Rn.op;
            s_len = Rn.len;
        }
        __syncthreads();
    }
    if (tid == 0) {
        Runs Rn{A.cigar + (uint64_t)qid * A.cigar_cap, A.cigar_cap, s_nops, s_op, s_len};
        const int i = s_i, k = s_k;
        Rn.emit(GWFA_CIGAR_EQ, (uint32_t)i);   // score 0: equal bases from (0, k)
        Rn.flush();
        o.walk_begin = (uint32_t)k;
        if (Rn.n <= Rn.cap)   // emitted end to start: reverse in place
            for (uint32_t a = 0, e = Rn.n; a + 1 < e; ++a, --e) {
                const uint32_t t = Rn.ops[a];
                Rn.ops[a] = Rn.ops[e - 1];
                Rn.ops[e - 1] = t;
            }
        o.cost = found;
        o.n_ops = Rn.n;
        o.status = Rn.n <= Rn.cap ? GWFA_OK : GWFA_ERR_CAPACITY;
        A.out[qid] = o;
    }
}

__global__ void __launch_bounds__(kThreads) cigar_kernel(CigarArgs A) {
    __shared__ uint32_t s_qid, s_base;
    __shared__ unsigned long long s_sum;
    __shared__ uint32_t s_warp[kThreads / 32];
    __shared__ int s_hitk;
    uint32_t *const tw = (uint32_t *)(A.ws + (uint64_t)blockIdx.x * A.ws_bytes);
    for (;;) {
        if (threadIdx.x == 0) s_qid = atomicAdd(A.head, 1u);
        __syncthreads();
        const uint32_t qid = s_qid;
        __syncthreads();
        if (qid >= A.n) return;
        align_walk(A, qid, tw, s_sum, s_warp, s_base, s_hitk);
        __syncthreads();
    }
}

}  // namespace

extern "C" int gwfa_cigar_create(const gwfa_graph *g, uint32_t ctas, uint64_t workspace_bytes,
                                 gwfa_cigar **out) {
    if (!g || !out) return GWFA_ERR_INVALID;
    *out = nullptr;
    if (cudaSetDevice(g->device) != cudaSuccess) return GWFA_ERR_CUDA;
    if (ctas == 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess)
            return GWFA_ERR_CUDA;
        ctas = 2u * (uint32_t)sms;
    }
    if (workspace_bytes == 0) workspace_bytes = 32ull << 20;
    workspace_bytes = (workspace_bytes + 255) & ~255ull;
    gwfa_cigar *c = new (std::nothrow) gwfa_cigar();
    if (!c) return GWFA_ERR_OOM;
    c->g = g;
    c->ctas = ctas;
    c->ws_bytes = workspace_bytes;
    if (cudaMalloc(&c->ws, workspace_bytes * ctas) != cudaSuccess ||
        cudaMalloc(&c->head, 256) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(c->ws);
        cudaFree(c->head);
        delete c;
        return GWFA_ERR_OOM;
    }
    *out = c;
    return GWFA_OK;
}

extern "C" int gwfa_cigar_destroy(gwfa_cigar *c) {
    if (!c) return GWFA_ERR_INVALID;
    cudaSetDevice(c->g->device);
    cudaFree(c->ws);
    cudaFree(c->head);
    delete c;
    return GWFA_OK;
}

extern "C" int gwfa_cigar_device(gwfa_cigar *c, uint32_t n_queries, const uint32_t *d_words,
                                 const uint64_t *d_q_off, const gwfa_result *d_res,
                                 const uint32_t *d_paths, uint32_t path_cap, const uint32_t *d_path_len,
                                 uint32_t *d_cigar, uint32_t cigar_cap, int32_t ends,
                                 gwfa_cigar_result *d_out, void *stream) {
    gwfa::Range range_("gwfa_cigar_device");
    if (!c || !d_words || !d_q_off || !d_res || !d_paths || !d_path_len || !d_out) return GWFA_ERR_INVALID;
    if (!d_cigar && cigar_cap) return GWFA_ERR_INVALID;
    if (path_cap == 0 || (ends & ~(GWFA_FREE_START | GWFA_FREE_END | GWFA_EXTEND))) return GWFA_ERR_INVALID;
    if (n_queries == 0) return GWFA_OK;
    if (cudaSetDevice(c->g->device) != cudaSuccess) return GWFA_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(c->head, 0, 4, s) != cudaSuccess) return GWFA_ERR_CUDA;
    CigarArgs a{};
    a.g = c->g->dev();
    a.qwords = d_words;
    a.q_off = d_q_off;
    a.res = d_res;
    a.paths = d_paths;
    a.path_cap = path_cap;
    a.path_len = d_path_len;
    a.cigar = d_cigar;
    a.cigar_cap = cigar_cap;
    a.out = d_out;
    a.ends = ends;
    a.ws = c->ws;
    a.ws_bytes = c->ws_bytes;
    a.n = n_queries;
    a.head = c->head;
    const uint32_t grid = c->ctas < n_queries ? c->ctas : n_queries;
    cigar_kernel<<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? GWFA_OK : GWFA_ERR_CUDA;
}
