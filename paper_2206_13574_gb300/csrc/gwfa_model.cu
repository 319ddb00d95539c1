// gwfa_model.cu -- learned cost model for scheduling batches of alignments.
//
// A tiny MLP (6 -> 32 -> 32 -> 4, ReLU) predicts, per query, log1p of: the edit
// distance (the number of scores of Alg. 1), the peak wavefront size, the
// number of diagonals that enter H~ (hash memory) and the total work (cells).
// It is trained on the work counters the alignment kernels report, never
// touches the alignment arithmetic, and is only used to order and place
// queries; a wrong prediction costs time (an overflow re-run), not accuracy.
//
// Numerics: FP16 weights and activations (inputs, hidden layers), FP32
// accumulation, FP32 master weights updated by Adam.  The network is small
// enough that one thread evaluates one sample; gradients are accumulated per
// block in shared memory and then atomically into global memory.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>
#include <unordered_map>
#include <utility>
#include <vector>

#include "gwfa_internal.cuh"

namespace {

constexpr int F = GWFA_MODEL_FEATURES;   // 6
constexpr int H = 32;
constexpr int O = GWFA_MODEL_TARGETS;    // 4
constexpr int NW1 = H * F, NB1 = H, NW2 = H * H, NB2 = H, NW3 = O * H, NB3 = O;
constexpr int OW1 = 0, OB1 = OW1 + NW1, OW2 = OB1 + NB1, OB2 = OW2 + NW2, OW3 = OB2 + NB2,
              OB3 = OW3 + NW3, NPARAM = OB3 + NB3;
static_assert(NPARAM == GWFA_MODEL_PARAMS, "parameter count");
constexpr int K = 16;       // k-mer length of the divergence feature
constexpr int SAMPLES = 64; // query k-mers sampled per query

// ---------------------------------------------------------------- features

struct FeatGraph {
    const uint32_t *kmers;   // sorted distinct 16-mers inside vertex labels (2-bit packed)
    uint64_t n_kmers;
    const uint4 *vinfo;      // {word, len, arc_begin, arc_end} as in the alignment kernels
    const uint32_t *arc_dst; // out-arc targets (CSR of the graph)
    const uint32_t *in_off;  // in-arcs: CSR by target, nv + 1
    const uint32_t *in_src;
    const uint8_t *arc_cyc;  // 1 for an out-arc inside a strongly connected component
    uint32_t nv;
};

// ---- the co-reachable subgraph of a query
//
// S = the vertices on some v_s -> v_e walk whose spelled length stays within the
// budget B = ceil(1.25 |q|) + 64 (the query's own walk spells about |q| bases;
// walks much longer than the query cannot be its alignment).  With f(v) = the
// shortest spelled length from v_s up to (not including) v and b(v) = the same from
// just after v to the end of v_e, v is in S iff f(v) + |v| + b(v) <= B.  Both are
// found by bounded label-correcting searches (forward from v_s, backward from v_e
// over in-arcs), whose result is the exact shortest lengths within the budget in
// any processing order.  The counts: |S|; arcs with both ends in S; vertices of S
// with two or more such arcs (bubble openings); such arcs inside a strongly
// connected component (loops).  A search that outgrows its table stops inserting
// and the counts cover what it reached.
constexpr uint32_t kSetCap = 8192;          // table entries per search (power of two)
constexpr uint32_t kSetLoad = kSetCap / 4 * 3;
constexpr uint32_t kFeatWarps = 1216;       // warps of the features kernel (8 per SM on 152 SMs)
constexpr uint32_t kEmptyV = 0xFFFFFFFFu;

__device__ __forceinline__ uint64_t feature_budget(uint64_t n) { return (5 * n + 3) / 4 + 64; }

// per-warp scratch: two tables (forward, backward) of (vertex, length) and two
// frontiers, in global memory
struct SetScratch {
    uint32_t *key[2], *dist[2], *fr[2];
};
__device__ __forceinline__ SetScratch set_scratch(uint32_t *base, uint32_t warp) {
    uint32_t *w = base + (uint64_t)warp * 6 * kSetCap;
    return SetScratch{{w, w + kSetCap}, {w + 2 * kSetCap, w + 3 * kSetCap}, {w + 4 * kSetCap, w + 5 * kSetCap}};
}

__device__ __forceinline__ uint32_t vhash(uint32_t v) { return (v * 0x9E3779B1u) & (kSetCap - 1); }

// slot of v in table t (inserted with length ~0 when absent), or -1 when full
__device__ int set_insert(const SetScratch &S, int t, uint32_t v, uint32_t *fill) {
    uint32_t h = vhash(v);
    for (uint32_t p = 0; p < kSetCap; ++p) {
        const uint32_t k = __ldcg(&S.key[t][h]);
        if (k == v) return (int)h;
        if (k == kEmptyV) {
            if (atomicAdd(fill, 0u) >= kSetLoad) return -1;
            const uint32_t prev = atomicCAS(&S.key[t][h], kEmptyV, v);
            if (prev == kEmptyV) {
                atomicAdd(fill, 1u);
                return (int)h;
            }
            if (prev == v) return (int)h;
        }
        h = (h + 1) & (kSetCap - 1);
    }
    return -1;
}
__device__ uint32_t set_find(const SetScratch &S, int t, uint32_t v) {
    uint32_t h = vhash(v);
    for (uint32_t p = 0; p < kSetCap; ++p) {
        const uint32_t k = __ldcg(&S.key[t][h]);
        if (k == v) return __ldcg(&S.dist[t][h]);
        if (k == kEmptyV) return kEmptyV;
        h = (h + 1) & (kSetCap - 1);
    }
    return kEmptyV;
}

// Bounded search of one warp: t = 0 forward from `src` over out-arcs, t = 1
// backward over in-arcs; lengths are spelled bases strictly before (forward) or
// after (backward) a vertex.
__device__ void bounded_search(const FeatGraph &fg, const SetScratch &S, int t, uint32_t src, uint64_t budget,
                               uint32_t *cnt /* shared: fill, frontier sizes [2] */) {
    const int lane = threadIdx.x & 31;
    for (uint32_t i = lane; i < kSetCap; i += 32) {
        __stcg(&S.key[t][i], kEmptyV);
        __stcg(&S.dist[t][i], kEmptyV);
    }
    if (lane == 0) {
        cnt[0] = 0;
        cnt[1] = 1;
        cnt[2] = 0;
    }
    __syncwarp();
    if (lane == 0) {
        const int h = set_insert(S, t, src, &cnt[0]);
        if (h >= 0) __stcg(&S.dist[t][h], 0u);
        __stcg(&S.fr[0][0], src);
    }
    __syncwarp();
    for (int cur = 0;; cur ^= 1) {
        const uint32_t nf = min(cnt[1 + cur], kSetCap);
        if (nf == 0) break;
        for (uint32_t i = lane; i < nf; i += 32) {
            const uint32_t v = __ldcg(&S.fr[cur][i]);
            const uint32_t dv = set_find(S, t, v);
            const uint4 vi = __ldg(&fg.vinfo[v]);
            // forward: a successor starts |v| bases later; backward: a predecessor u
            // ends where v starts, so its length after it is b(v) + |v|
            const uint64_t cand = (uint64_t)dv + vi.y;
            if (cand > budget) continue;
            const uint32_t a0 = t == 0 ? vi.z : __ldg(&fg.in_off[v]);
            const uint32_t a1 = t == 0 ? vi.w : __ldg(&fg.in_off[v + 1]);
            for (uint32_t a = a0; a < a1; ++a) {
                const uint32_t u = t == 0 ? __ldg(&fg.arc_dst[a]) : __ldg(&fg.in_src[a]);
                const int h = set_insert(S, t, u, &cnt[0]);
                if (h < 0) continue;
                if (atomicMin(&S.dist[t][h], (uint32_t)cand) > (uint32_t)cand) {
                    const uint32_t k = atomicAdd(&cnt[2 - cur], 1u);
                    if (k < kSetCap) __stcg(&S.fr[cur ^ 1][k], u);
                }
            }
        }
        __syncwarp();
        if (lane == 0) cnt[1 + cur] = 0;
        __syncwarp();
    }
}

__device__ __forceinline__ uint32_t qwindow16(const uint32_t *w, uint64_t p) {
    const uint64_t wi = p >> 4;
    const uint32_t sh = (uint32_t)(p & 15) * 2;
    return __funnelshift_r(__ldg(w + wi), __ldg(w + wi + 1), sh);
}

__device__ bool kmer_present(const uint32_t *a, uint64_t n, uint32_t key) {
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        const uint32_t x = __ldg(a + mid);
        if (x < key) lo = mid + 1;
        else hi = mid;
    }
    return lo < n && __ldg(a + lo) == key;
}

// Raw features of each query (one warp per query, two sampled k-mers per lane):
//   0 log1p(|q|)
//   1 fraction of 64 evenly spaced query 16-mers absent from the graph's labels
//   2 log1p(|S|), S the co-reachable subgraph above
//   3 log1p(arcs inside S)
//   4 vertices of S with two or more arcs inside S, per kb of query
//   5 log1p(arcs inside S that lie on a cycle)
__global__ void features_kernel(FeatGraph fg, uint32_t nq, const uint32_t *__restrict__ words,
                                const uint64_t *__restrict__ q_off, const uint32_t *__restrict__ vs,
                                const uint32_t *__restrict__ ve, float *__restrict__ feat,
                                uint32_t *__restrict__ scratch) {
    __shared__ uint32_t s_cnt[8][3];
    const int lane = threadIdx.x & 31;
    const uint32_t wpb = blockDim.x >> 5;
    const uint32_t wib = threadIdx.x >> 5;
    const SetScratch S = set_scratch(scratch, blockIdx.x * wpb + wib);
    for (uint32_t qi = blockIdx.x * wpb + wib; qi < nq; qi += gridDim.x * wpb) {
        const uint64_t qo = q_off[qi];
        const uint64_t n = q_off[qi + 1] - qo;
        const uint32_t *qw = words + (qo >> 4) + qi;
        int miss = 0;
        if (n >= K) {
            for (int t = lane; t < SAMPLES; t += 32) {
                const uint64_t p = (uint64_t)t * (n - K) / (SAMPLES - 1);
                miss += kmer_present(fg.kmers, fg.n_kmers, qwindow16(qw, p)) ? 0 : 1;
            }
        }
        for (int o = 16; o >= 1; o >>= 1) miss += __shfl_xor_sync(0xFFFFFFFFu, miss, o);
        // the co-reachable subgraph
        const uint32_t a = min(vs[qi], fg.nv - 1), b = min(ve[qi], fg.nv - 1);
        const uint64_t budget = feature_budget(n);
        bounded_search(fg, S, 0, a, budget, s_cnt[wib]);
        bounded_search(fg, S, 1, b, budget, s_cnt[wib]);
        uint32_t nverts = 0, narcs = 0, nbub = 0, ncyc = 0;
        for (uint32_t i = lane; i < kSetCap; i += 32) {
            const uint32_t v = __ldcg(&S.key[0][i]);
            if (v == kEmptyV) continue;
            const uint32_t fv = __ldcg(&S.dist[0][i]), bv = set_find(S, 1, v);
            const uint4 vi = __ldg(&fg.vinfo[v]);
            if (bv == kEmptyV || (uint64_t)fv + vi.y + bv > budget) continue;
            ++nverts;
            uint32_t deg = 0;
            for (uint32_t e = vi.z; e < vi.w; ++e) {
                const uint32_t u = __ldg(&fg.arc_dst[e]);
                const uint32_t fu = set_find(S, 0, u), bu = set_find(S, 1, u);
                if (fu == kEmptyV || bu == kEmptyV || (uint64_t)fu + __ldg(&fg.vinfo[u]).y + bu > budget) continue;
                ++deg;
                ncyc += __ldg(&fg.arc_cyc[e]);
            }
            narcs += deg;
            nbub += deg > 1 ? 1u : 0u;
        }
        nverts = __reduce_add_sync(0xFFFFFFFFu, nverts);
        narcs = __reduce_add_sync(0xFFFFFFFFu, narcs);
        nbub = __reduce_add_sync(0xFFFFFFFFu, nbub);
        ncyc = __reduce_add_sync(0xFFFFFFFFu, ncyc);
        if (lane == 0) {
            float *f = feat + (uint64_t)qi * F;
            f[0] = log1pf((float)n);
            f[1] = n >= K ? (float)miss / SAMPLES : 0.f;
            f[2] = log1pf((float)nverts);
            f[3] = log1pf((float)narcs);
            f[4] = (float)nbub * 1000.f / (float)max(n, (uint64_t)1);
            f[5] = log1pf((float)ncyc);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- MLP

struct Norm {
    float fmean[F], fstd[F], tmean[O], tstd[O];
};

// one sample forward: FP16 inputs / activations / weights, FP32 accumulation
__device__ __forceinline__ void mlp_forward(const __half *__restrict__ w, const Norm &nm,
                                            const float *__restrict__ f, __half xs[F], __half h1[H],
                                            __half h2[H], float out[O]) {
    for (int i = 0; i < F; ++i) xs[i] = __float2half((f[i] - nm.fmean[i]) / nm.fstd[i]);
    for (int o = 0; o < H; ++o) {
        float acc = __half2float(w[OB1 + o]);
        for (int i = 0; i < F; ++i) acc = fmaf(__half2float(w[OW1 + o * F + i]), __half2float(xs[i]), acc);
        h1[o] = __float2half(fmaxf(acc, 0.f));
    }
    for (int o = 0; o < H; ++o) {
        float acc = __half2float(w[OB2 + o]);
        for (int i = 0; i < H; ++i) acc = fmaf(__half2float(w[OW2 + o * H + i]), __half2float(h1[i]), acc);
        h2[o] = __float2half(fmaxf(acc, 0.f));
    }
    for (int o = 0; o < O; ++o) {
        float acc = __half2float(w[OB3 + o]);
        for (int i = 0; i < H; ++i) acc = fmaf(__half2float(w[OW3 + o * H + i]), __half2float(h2[i]), acc);
        out[o] = acc;   // normalised target units
    }
}

__global__ void predict_kernel(const __half *__restrict__ w16, Norm nm, uint32_t n,
                               const float *__restrict__ feat, float *__restrict__ pred) {
    __shared__ __half w[NPARAM];
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) w[i] = w16[i];
    __syncthreads();
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        __half xs[F], h1[H], h2[H];
        float out[O];
        mlp_forward(w, nm, feat + (uint64_t)s * F, xs, h1, h2, out);
        for (int o = 0; o < O; ++o) pred[(uint64_t)s * O + o] = out[o] * nm.tstd[o] + nm.tmean[o];
    }
}

// Forward + backward of the mean squared error over `count` samples
// (index list `idx`, or 0..count-1 when NULL), gradient summed into g (fp32),
// loss summed into *loss.  dL/dout = 2 (out - y) / (count * O).
__global__ void grad_kernel(const __half *__restrict__ w16, Norm nm, uint32_t count,
                            const uint32_t *__restrict__ idx, const float *__restrict__ feat,
                            const float *__restrict__ target, float *__restrict__ g,
                            float *__restrict__ loss) {
    __shared__ __half w[NPARAM];
    __shared__ float gs[NPARAM];
    __shared__ float ls;
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) {
        w[i] = w16[i];
        gs[i] = 0.f;
    }
    if (threadIdx.x == 0) ls = 0.f;
    __syncthreads();
    const float scale = 2.f / ((float)count * O);
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
        const uint32_t s = idx ? idx[t] : t;
        __half xs[F], h1[H], h2[H];
        float out[O], gout[O];
        mlp_forward(w, nm, feat + (uint64_t)s * F, xs, h1, h2, out);
        float l = 0.f;
        for (int o = 0; o < O; ++o) {
            const float y = (target[(uint64_t)s * O + o] - nm.tmean[o]) / nm.tstd[o];
            const float e = out[o] - y;
            l += e * e;
            gout[o] = scale * e;
        }
        atomicAdd(&ls, l / ((float)count * O));
        // layer 3
        float ga2[H];
        for (int i = 0; i < H; ++i) ga2[i] = 0.f;
        for (int o = 0; o < O; ++o) {
            atomicAdd(&gs[OB3 + o], gout[o]);
            for (int i = 0; i < H; ++i) {
                atomicAdd(&gs[OW3 + o * H + i], gout[o] * __half2float(h2[i]));
                ga2[i] += gout[o] * __half2float(w[OW3 + o * H + i]);
            }
        }
        for (int i = 0; i < H; ++i) ga2[i] = __half2float(h2[i]) > 0.f ? ga2[i] : 0.f;
        // layer 2
        float ga1[H];
        for (int i = 0; i < H; ++i) ga1[i] = 0.f;
        for (int o = 0; o < H; ++o) {
            if (ga2[o] == 0.f) continue;
            atomicAdd(&gs[OB2 + o], ga2[o]);
            for (int i = 0; i < H; ++i) {
                atomicAdd(&gs[OW2 + o * H + i], ga2[o] * __half2float(h1[i]));
                ga1[i] += ga2[o] * __half2float(w[OW2 + o * H + i]);
            }
        }
        // layer 1
        for (int o = 0; o < H; ++o) {
            const float ga = __half2float(h1[o]) > 0.f ? ga1[o] : 0.f;
            if (ga == 0.f) continue;
            atomicAdd(&gs[OB1 + o], ga);
            for (int i = 0; i < F; ++i) atomicAdd(&gs[OW1 + o * F + i], ga * __half2float(xs[i]));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x)
        if (gs[i] != 0.f) atomicAdd(&g[i], gs[i]);
    if (threadIdx.x == 0) atomicAdd(loss, ls);
}

// Adam on the FP32 master weights, then the FP16 copy used by the kernels.
__global__ void adam_kernel(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                            float *__restrict__ g, __half *__restrict__ w16, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    w16[i] = __float2half(wi);
    g[i] = 0.f;   // ready for the next step
}

__global__ void to_half_kernel(const float *__restrict__ w, __half *__restrict__ w16, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w16[i] = __float2half(w[i]);
}

int cstat(cudaError_t e) {
    if (e == cudaSuccess) return GWFA_OK;
    return e == cudaErrorMemoryAllocation ? GWFA_ERR_OOM : GWFA_ERR_CUDA;
}

uint64_t splitmix(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

struct gwfa_model {
    const gwfa_graph *g = nullptr;
    // host copies for predicting single requests on the host (serving admission)
    std::vector<uint32_t> h_kmers, h_in_off, h_in_src;
    std::vector<uint8_t> h_arc_cyc;
    std::vector<float> h_w;
    FeatGraph fg{};
    uint32_t *d_kmers = nullptr, *d_in_off = nullptr, *d_in_src = nullptr, *d_scratch = nullptr;
    uint8_t *d_arc_cyc = nullptr;
    float *d_w = nullptr, *d_m = nullptr, *d_v = nullptr, *d_g = nullptr, *d_loss = nullptr;
    __half *d_w16 = nullptr;
    uint32_t *d_idx = nullptr;
    uint64_t idx_cap = 0;
    Norm norm{};
    uint64_t adam_t = 0;
    cudaStream_t stream = nullptr;
    std::mutex mu;
};

// Strongly connected components (iterative Tarjan): component id per vertex.
static std::vector<uint32_t> strong_components(uint32_t nv, const std::vector<uint32_t> &off,
                                        const std::vector<uint32_t> &dst) {
    const uint32_t none = 0xFFFFFFFFu;
    std::vector<uint32_t> index(nv, none), low(nv, 0), comp(nv, none), stack;
    std::vector<uint8_t> on(nv, 0);
    std::vector<std::pair<uint32_t, uint32_t>> call;   // (vertex, next arc)
    uint32_t next_index = 0, next_comp = 0;
    for (uint32_t r = 0; r < nv; ++r) {
        if (index[r] != none) continue;
        call.push_back({r, off[r]});
        index[r] = low[r] = next_index++;
        stack.push_back(r);
        on[r] = 1;
        while (!call.empty()) {
            const uint32_t v = call.back().first;
            uint32_t &a = call.back().second;
            if (a < off[v + 1]) {
                const uint32_t w = dst[a++];
                if (index[w] == none) {
                    index[w] = low[w] = next_index++;
                    stack.push_back(w);
                    on[w] = 1;
                    call.push_back({w, off[w]});
                } else if (on[w]) {
                    low[v] = std::min(low[v], index[w]);
                }
                continue;
            }
            call.pop_back();
            if (!call.empty()) low[call.back().first] = std::min(low[call.back().first], low[v]);
            if (low[v] == index[v]) {
                uint32_t w;
                do {
                    w = stack.back();
                    stack.pop_back();
                    on[w] = 0;
                    comp[w] = next_comp;
                } while (w != v);
                ++next_comp;
            }
        }
    }
    return comp;
}

// vertex -> spelled length, open addressing (the host searches run once per served
// request, so they avoid node allocation)
struct DistMap {
    std::vector<uint32_t> key;
    std::vector<uint64_t> val;
    uint32_t mask = 0, size = 0;
    static constexpr uint32_t kEmpty = 0xFFFFFFFFu;
    DistMap() : key(1024, kEmpty), val(1024, 0), mask(1023) {}
    uint32_t slot(uint32_t v) const {
        uint32_t h = (v * 0x9E3779B1u) & mask;
        while (key[h] != kEmpty && key[h] != v) h = (h + 1) & mask;
        return h;
    }
    const uint64_t *find(uint32_t v) const {
        const uint32_t h = slot(v);
        return key[h] == v ? &val[h] : nullptr;
    }
    // sets v's length to d if absent or larger; true if it changed
    bool lower(uint32_t v, uint64_t d) {
        uint32_t h = slot(v);
        if (key[h] == v) {
            if (d >= val[h]) return false;
            val[h] = d;
            return true;
        }
        if (2 * (size + 1) > mask + 1) {   // keep the load at most one half
            std::vector<uint32_t> k2;
            std::vector<uint64_t> v2;
            k2.swap(key);
            v2.swap(val);
            key.assign(2 * k2.size(), kEmpty);
            val.assign(2 * k2.size(), 0);
            mask = (uint32_t)key.size() - 1;
            for (size_t i = 0; i < k2.size(); ++i)
                if (k2[i] != kEmpty) {
                    const uint32_t s2 = slot(k2[i]);
                    key[s2] = k2[i];
                    val[s2] = v2[i];
                }
            h = slot(v);
        }
        key[h] = v;
        val[h] = d;
        ++size;
        return true;
    }
};

// The co-reachable subgraph counts of the features kernel, on the host (serving
// admission): |S|, arcs inside S, vertices with two or more of them, cycle arcs.
static void coreachable_counts(const gwfa_model *m, uint32_t vs, uint32_t ve, uint64_t n, uint32_t out[4]) {
    const gwfa_graph *g = m->g;
    const uint64_t budget = (5 * n + 3) / 4 + 64;
    auto len = [&](uint32_t v) { return (uint64_t)(g->h_vlen[v]); };
    auto search = [&](uint32_t src, bool fwd, DistMap &dist) {
        std::vector<uint32_t> cur{src}, nxt;
        dist.lower(src, 0);
        while (!cur.empty()) {
            nxt.clear();
            for (uint32_t v : cur) {
                const uint64_t c = *dist.find(v) + len(v);
                if (c > budget) continue;
                const uint32_t a0 = fwd ? g->h_arc_off[v] : m->h_in_off[v];
                const uint32_t a1 = fwd ? g->h_arc_off[v + 1] : m->h_in_off[v + 1];
                for (uint32_t a = a0; a < a1; ++a) {
                    const uint32_t u = fwd ? g->h_arc_dst[a] : m->h_in_src[a];
                    if (dist.lower(u, c)) nxt.push_back(u);
                }
            }
            std::swap(cur, nxt);
        }
    };
    DistMap f, b;
    search(vs, true, f);
    search(ve, false, b);
    auto in_s = [&](uint32_t v) {
        const uint64_t *i = f.find(v), *j = b.find(v);
        return i && j && *i + len(v) + *j <= budget;
    };
    uint32_t nverts = 0, narcs = 0, nbub = 0, ncyc = 0;
    for (size_t x = 0; x < f.key.size(); ++x) {
        const uint32_t v = f.key[x];
        if (v == DistMap::kEmpty || !in_s(v)) continue;
        ++nverts;
        uint32_t deg = 0;
        for (uint32_t a = g->h_arc_off[v]; a < g->h_arc_off[v + 1]; ++a) {
            if (!in_s(g->h_arc_dst[a])) continue;
            ++deg;
            ncyc += m->h_arc_cyc[a];
        }
        narcs += deg;
        nbub += deg > 1 ? 1 : 0;
    }
    out[0] = nverts;
    out[1] = narcs;
    out[2] = nbub;
    out[3] = ncyc;
}

extern "C" {

int gwfa_model_create(const gwfa_graph *g, uint64_t seed, gwfa_model **out) {
    if (!g || !out) return GWFA_ERR_INVALID;
    *out = nullptr;
    int st = cstat(cudaSetDevice(g->device));
    if (st) return st;
    // graph-side feature tables, from the host copy of the graph
    std::vector<uint32_t> words(g->n_words);
    std::vector<uint4> vinfo(g->nv);
    if (cudaMemcpy(words.data(), g->d_words, g->n_words * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(vinfo.data(), g->d_vinfo, (uint64_t)g->nv * sizeof(uint4), cudaMemcpyDeviceToHost) !=
            cudaSuccess)
        return GWFA_ERR_CUDA;
    std::vector<uint32_t> kmers;
    kmers.reserve(g->total);
    for (uint32_t v = 0; v < g->nv; ++v) {
        const uint32_t w0 = vinfo[v].x, L = vinfo[v].y;
        for (uint32_t p = 0; p + K <= L; ++p) {
            const uint64_t pos = (uint64_t)w0 * 16 + p, wi = pos >> 4;
            const uint32_t sh = (uint32_t)(pos & 15) * 2;
            const uint64_t two = (uint64_t)words[wi] | ((uint64_t)words[wi + 1] << 32);
            kmers.push_back((uint32_t)(two >> sh));
        }
    }
    std::sort(kmers.begin(), kmers.end());
    kmers.erase(std::unique(kmers.begin(), kmers.end()), kmers.end());
    // in-arcs (CSR by target) for the backward search, and which arcs lie on a cycle
    const uint64_t na = g->h_arc_dst.size();
    std::vector<uint32_t> in_off(g->nv + 1, 0), in_src(na);
    for (uint64_t a = 0; a < na; ++a) in_off[g->h_arc_dst[a] + 1]++;
    for (uint32_t v = 0; v < g->nv; ++v) in_off[v + 1] += in_off[v];
    {
        std::vector<uint32_t> pos(in_off.begin(), in_off.end() - 1);
        for (uint32_t v = 0; v < g->nv; ++v)
            for (uint32_t a = g->h_arc_off[v]; a < g->h_arc_off[v + 1]; ++a) in_src[pos[g->h_arc_dst[a]]++] = v;
    }
    const std::vector<uint32_t> comp = strong_components(g->nv, g->h_arc_off, g->h_arc_dst);
    std::vector<uint8_t> arc_cyc(std::max<uint64_t>(na, 1), 0);
    for (uint32_t v = 0; v < g->nv; ++v)
        for (uint32_t a = g->h_arc_off[v]; a < g->h_arc_off[v + 1]; ++a)
            arc_cyc[a] = comp[v] == comp[g->h_arc_dst[a]] ? 1 : 0;
    gwfa_model *m = new (std::nothrow) gwfa_model();
    if (!m) return GWFA_ERR_OOM;
    m->g = g;
    st = cstat(cudaMalloc(&m->d_kmers, std::max<uint64_t>(kmers.size(), 1) * 4));
    if (!st) st = cstat(cudaMalloc(&m->d_in_off, (uint64_t)(g->nv + 1) * 4));
    if (!st) st = cstat(cudaMalloc(&m->d_in_src, std::max<uint64_t>(na, 1) * 4));
    if (!st) st = cstat(cudaMalloc(&m->d_arc_cyc, arc_cyc.size()));
    if (!st) st = cstat(cudaMalloc(&m->d_scratch, (uint64_t)kFeatWarps * 6 * kSetCap * 4));
    if (!st) st = cstat(cudaMalloc(&m->d_w, NPARAM * 4));
    if (!st) st = cstat(cudaMalloc(&m->d_m, NPARAM * 4));
    if (!st) st = cstat(cudaMalloc(&m->d_v, NPARAM * 4));
    if (!st) st = cstat(cudaMalloc(&m->d_g, NPARAM * 4));
    if (!st) st = cstat(cudaMalloc(&m->d_loss, 64));
    if (!st) st = cstat(cudaMalloc(&m->d_w16, NPARAM * 2));
    if (!st) st = cstat(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking));
    if (!st && !kmers.empty())
        st = cstat(cudaMemcpy(m->d_kmers, kmers.data(), kmers.size() * 4, cudaMemcpyHostToDevice));
    if (!st) st = cstat(cudaMemcpy(m->d_in_off, in_off.data(), in_off.size() * 4, cudaMemcpyHostToDevice));
    if (!st && na) st = cstat(cudaMemcpy(m->d_in_src, in_src.data(), na * 4, cudaMemcpyHostToDevice));
    if (!st) st = cstat(cudaMemcpy(m->d_arc_cyc, arc_cyc.data(), arc_cyc.size(), cudaMemcpyHostToDevice));
    if (st) { gwfa_model_destroy(m); return st; }
    m->fg = FeatGraph{m->d_kmers, kmers.size(), g->d_vinfo, g->d_arc_dst, m->d_in_off, m->d_in_src,
                      m->d_arc_cyc, g->nv};
    m->h_kmers = std::move(kmers);
    m->h_in_off = std::move(in_off);
    m->h_in_src = std::move(in_src);
    m->h_arc_cyc = std::move(arc_cyc);
    // He-style initialisation from a seeded SplitMix64 stream
    std::vector<float> w(NPARAM, 0.f);
    uint64_t s = seed;
    auto uni = [&]() { return (float)((splitmix(s) >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f; };
    for (int i = 0; i < NW1; ++i) w[OW1 + i] = uni() * std::sqrt(6.f / F);
    for (int i = 0; i < NW2; ++i) w[OW2 + i] = uni() * std::sqrt(6.f / H);
    for (int i = 0; i < NW3; ++i) w[OW3 + i] = uni() * std::sqrt(3.f / H);
    for (int i = 0; i < F; ++i) { m->norm.fmean[i] = 0.f; m->norm.fstd[i] = 1.f; }
    for (int i = 0; i < O; ++i) { m->norm.tmean[i] = 0.f; m->norm.tstd[i] = 1.f; }
    st = gwfa_model_set_params(m, w.data(), NPARAM);
    if (st) { gwfa_model_destroy(m); return st; }
    *out = m;
    return GWFA_OK;
}

int gwfa_model_destroy(gwfa_model *m) {
    if (!m) return GWFA_ERR_INVALID;
    cudaSetDevice(m->g->device);
    cudaFree(m->d_kmers);
    cudaFree(m->d_in_off);
    cudaFree(m->d_in_src);
    cudaFree(m->d_arc_cyc);
    cudaFree(m->d_scratch);
    cudaFree(m->d_w);
    cudaFree(m->d_m);
    cudaFree(m->d_v);
    cudaFree(m->d_g);
    cudaFree(m->d_loss);
    cudaFree(m->d_w16);
    cudaFree(m->d_idx);
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
    return GWFA_OK;
}

int gwfa_model_set_params(gwfa_model *m, const float *h_params, uint32_t n_params) {
    if (!m || !h_params || n_params != NPARAM) return GWFA_ERR_INVALID;
    std::lock_guard<std::mutex> lk(m->mu);
    int st = cstat(cudaSetDevice(m->g->device));
    if (!st) st = cstat(cudaMemcpy(m->d_w, h_params, NPARAM * 4, cudaMemcpyHostToDevice));
    if (!st) st = cstat(cudaMemset(m->d_m, 0, NPARAM * 4));
    if (!st) st = cstat(cudaMemset(m->d_v, 0, NPARAM * 4));
    if (!st) st = cstat(cudaMemset(m->d_g, 0, NPARAM * 4));
    if (!st) {
        to_half_kernel<<<(NPARAM + 255) / 256, 256>>>(m->d_w, m->d_w16, NPARAM);
        st = cstat(cudaGetLastError());
    }
    if (!st) st = cstat(cudaDeviceSynchronize());
    m->adam_t = 0;
    if (!st) m->h_w.assign(h_params, h_params + NPARAM);
    return st;
}

int gwfa_model_get_params(const gwfa_model *m, float *h_params, uint32_t n_params) {
    if (!m || !h_params || n_params != NPARAM) return GWFA_ERR_INVALID;
    if (cudaSetDevice(m->g->device) != cudaSuccess) return GWFA_ERR_CUDA;
    return cstat(cudaMemcpy(h_params, m->d_w, NPARAM * 4, cudaMemcpyDeviceToHost));
}

int gwfa_model_set_normalization(gwfa_model *m, const float *fmean, const float *fstd,
                                 const float *tmean, const float *tstd) {
    if (!m || !fmean || !fstd || !tmean || !tstd) return GWFA_ERR_INVALID;
    for (int i = 0; i < F; ++i)
        if (!(fstd[i] > 0.f)) return GWFA_ERR_INVALID;
    for (int i = 0; i < O; ++i)
        if (!(tstd[i] > 0.f)) return GWFA_ERR_INVALID;
    std::lock_guard<std::mutex> lk(m->mu);
    memcpy(m->norm.fmean, fmean, sizeof(m->norm.fmean));
    memcpy(m->norm.fstd, fstd, sizeof(m->norm.fstd));
    memcpy(m->norm.tmean, tmean, sizeof(m->norm.tmean));
    memcpy(m->norm.tstd, tstd, sizeof(m->norm.tstd));
    return GWFA_OK;
}

// Model file: 8-byte tag, the parameter / feature / target counts (uint32 each), then
// the fp32 parameters and the four normalisation vectors, host byte order.
static const char kModelTag[8] = {'G', 'W', 'F', 'A', 'M', 'L', 'P', '1'};

int gwfa_model_save(const gwfa_model *m, const char *path) {
    if (!m || !path) return GWFA_ERR_INVALID;
    std::vector<float> w(NPARAM);
    int st = gwfa_model_get_params(m, w.data(), NPARAM);
    if (st) return st;
    Norm nm;
    {
        std::lock_guard<std::mutex> lk(const_cast<gwfa_model *>(m)->mu);
        nm = m->norm;
    }
    FILE *f = fopen(path, "wb");
    if (!f) return GWFA_ERR_INVALID;
    const uint32_t dims[3] = {(uint32_t)NPARAM, (uint32_t)F, (uint32_t)O};
    bool ok = fwrite(kModelTag, 1, 8, f) == 8 && fwrite(dims, 4, 3, f) == 3 &&
              fwrite(w.data(), 4, NPARAM, f) == (size_t)NPARAM && fwrite(&nm, sizeof(nm), 1, f) == 1;
    ok = (fclose(f) == 0) && ok;
    return ok ? GWFA_OK : GWFA_ERR_INVALID;
}

int gwfa_model_load(gwfa_model *m, const char *path) {
    if (!m || !path) return GWFA_ERR_INVALID;
    FILE *f = fopen(path, "rb");
    if (!f) return GWFA_ERR_INVALID;
    char tag[8];
    uint32_t dims[3];
    std::vector<float> w(NPARAM);
    Norm nm;
    bool ok = fread(tag, 1, 8, f) == 8 && memcmp(tag, kModelTag, 8) == 0 && fread(dims, 4, 3, f) == 3 &&
              dims[0] == (uint32_t)NPARAM && dims[1] == (uint32_t)F && dims[2] == (uint32_t)O &&
              fread(w.data(), 4, NPARAM, f) == (size_t)NPARAM && fread(&nm, sizeof(nm), 1, f) == 1;
    fclose(f);
    if (!ok) return GWFA_ERR_INVALID;
    int st = gwfa_model_set_normalization(m, nm.fmean, nm.fstd, nm.tmean, nm.tstd);
    if (!st) st = gwfa_model_set_params(m, w.data(), NPARAM);
    return st;
}

int gwfa_model_features_device(gwfa_model *m, uint32_t n, const uint32_t *d_words,
                               const uint64_t *d_q_off, const uint32_t *d_v_s, const uint32_t *d_v_e,
                               float *d_feat, void *stream) {
    if (!m || !d_words || !d_q_off || !d_v_s || !d_v_e || !d_feat) return GWFA_ERR_INVALID;
    if (n == 0) return GWFA_OK;
    int st = cstat(cudaSetDevice(m->g->device));
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;   // NULL = the legacy default stream
    // kFeatWarps warps (8 per CTA), each with its own search tables in d_scratch
    const uint32_t blocks = std::min<uint32_t>((n + 7) / 8, kFeatWarps / 8);
    features_kernel<<<blocks, 256, 0, s>>>(m->fg, n, d_words, d_q_off, d_v_s, d_v_e, d_feat, m->d_scratch);
    return cstat(cudaGetLastError());
}

int gwfa_model_predict_device(gwfa_model *m, uint32_t n, const float *d_feat, float *d_pred,
                              void *stream) {
    if (!m || !d_feat || !d_pred) return GWFA_ERR_INVALID;
    if (n == 0) return GWFA_OK;
    int st = cstat(cudaSetDevice(m->g->device));
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;   // NULL = the legacy default stream
    const uint32_t blocks = std::min<uint32_t>((n + 255) / 256, 1024);
    predict_kernel<<<blocks, 256, 0, s>>>(m->d_w16, m->norm, n, d_feat, d_pred);
    return cstat(cudaGetLastError());
}

int gwfa_model_gradient_device(gwfa_model *m, uint32_t n, const float *d_feat, const float *d_target,
                               float *h_grad, float *h_loss, void *stream) {
    if (!m || !d_feat || !d_target || !h_grad || n == 0) return GWFA_ERR_INVALID;
    std::lock_guard<std::mutex> lk(m->mu);
    int st = cstat(cudaSetDevice(m->g->device));
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;   // NULL = the legacy default stream
    st = cstat(cudaMemsetAsync(m->d_g, 0, NPARAM * 4, s));
    if (!st) st = cstat(cudaMemsetAsync(m->d_loss, 0, 4, s));
    if (st) return st;
    const uint32_t blocks = std::min<uint32_t>((n + 127) / 128, 512);
    grad_kernel<<<blocks, 128, 0, s>>>(m->d_w16, m->norm, n, nullptr, d_feat, d_target, m->d_g, m->d_loss);
    st = cstat(cudaGetLastError());
    if (!st) st = cstat(cudaMemcpyAsync(h_grad, m->d_g, NPARAM * 4, cudaMemcpyDeviceToHost, s));
    if (!st && h_loss) st = cstat(cudaMemcpyAsync(h_loss, m->d_loss, 4, cudaMemcpyDeviceToHost, s));
    if (!st) st = cstat(cudaMemsetAsync(m->d_g, 0, NPARAM * 4, s));
    if (!st) st = cstat(cudaStreamSynchronize(s));
    return st;
}

int gwfa_model_train_device(gwfa_model *m, uint32_t n, const float *d_feat, const float *d_target,
                            uint32_t steps, uint32_t batch, float lr, uint64_t seed, float *h_losses,
                            void *stream) {
    gwfa::Range range_("gwfa_model_train_device");
    if (!m || !d_feat || !d_target || n == 0 || steps == 0 || batch == 0 || !(lr > 0.f))
        return GWFA_ERR_INVALID;
    std::lock_guard<std::mutex> lk(m->mu);
    int st = cstat(cudaSetDevice(m->g->device));
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;   // NULL = the legacy default stream
    batch = std::min(batch, n);
    // minibatch index lists: consecutive slices of seeded permutations, on the device
    const uint64_t total = (uint64_t)steps * batch;
    if (m->idx_cap < total) {
        cudaFree(m->d_idx);
        m->d_idx = nullptr;
        m->idx_cap = 0;
        st = cstat(cudaMalloc(&m->d_idx, total * 4));
        if (st) return st;
        m->idx_cap = total;
    }
    std::vector<uint32_t> perm(n), idx(total);
    uint64_t rs = seed;
    uint64_t k = 0;
    while (k < total) {
        for (uint32_t i = 0; i < n; ++i) perm[i] = i;
        for (uint32_t i = n - 1; i > 0; --i) std::swap(perm[i], perm[splitmix(rs) % (i + 1)]);
        for (uint32_t i = 0; i < n && k < total; ++i) idx[k++] = perm[i];
    }
    st = cstat(cudaMemcpyAsync(m->d_idx, idx.data(), total * 4, cudaMemcpyHostToDevice, s));
    if (!st) st = cstat(cudaMemsetAsync(m->d_g, 0, NPARAM * 4, s));
    if (!st) st = cstat(cudaMemsetAsync(m->d_loss, 0, 64, s));
    if (st) return st;
    std::vector<float> losses;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const uint32_t blocks = std::min<uint32_t>((batch + 127) / 128, 256);
    for (uint32_t t = 0; t < steps; ++t) {
        grad_kernel<<<blocks, 128, 0, s>>>(m->d_w16, m->norm, batch, m->d_idx + (uint64_t)t * batch,
                                           d_feat, d_target, m->d_g, m->d_loss + (t & 7));
        ++m->adam_t;
        const float c1 = 1.f - std::pow(b1, (float)m->adam_t), c2 = 1.f - std::pow(b2, (float)m->adam_t);
        adam_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(m->d_w, m->d_m, m->d_v, m->d_g, m->d_w16, lr, b1,
                                                        b2, eps, c1, c2);
        st = cstat(cudaGetLastError());
        if (st) return st;
        if (h_losses && ((t & 7) == 7 || t + 1 == steps)) {
            float l8[8];
            st = cstat(cudaMemcpyAsync(l8, m->d_loss, 32, cudaMemcpyDeviceToHost, s));
            if (!st) st = cstat(cudaMemsetAsync(m->d_loss, 0, 32, s));
            if (!st) st = cstat(cudaStreamSynchronize(s));
            if (st) return st;
            for (uint32_t j = t - (t & 7); j <= t; ++j) h_losses[j] = l8[j & 7];
        }
    }
    st = cstat(cudaStreamSynchronize(s));
    if (!st) {
        m->h_w.resize(NPARAM);
        st = cstat(cudaMemcpy(m->h_w.data(), m->d_w, NPARAM * 4, cudaMemcpyDeviceToHost));
    }
    return st;
}

int gwfa_model_predict_host(const gwfa_model *m, const char *q, uint32_t n, uint32_t v_s, uint32_t v_e,
                            float *h_pred) {
    if (!m || !h_pred || (n && !q) || m->h_w.size() != (size_t)NPARAM) return GWFA_ERR_INVALID;
    const uint32_t nv = m->g->nv;
    if (v_s >= nv || v_e >= nv) return GWFA_ERR_INVALID;
    // the same six features as features_kernel, from the ASCII query
    std::vector<uint8_t> c(n);
    for (uint32_t i = 0; i < n; ++i) {
        const char ch = q[i];
        c[i] = (ch == 'C' || ch == 'c') ? 1 : (ch == 'G' || ch == 'g') ? 2 : (ch == 'T' || ch == 't') ? 3 : 0;
    }
    int miss = 0;
    if (n >= (uint32_t)K) {
        for (int t = 0; t < SAMPLES; ++t) {
            const uint64_t p = (uint64_t)t * (n - K) / (SAMPLES - 1);
            uint32_t key = 0;
            for (int b = 0; b < K; ++b) key |= (uint32_t)c[p + b] << (2 * b);
            miss += std::binary_search(m->h_kmers.begin(), m->h_kmers.end(), key) ? 0 : 1;
        }
    }
    uint32_t sub[4];
    coreachable_counts(m, v_s, v_e, n, sub);
    const float f[F] = {std::log1p((float)n), n >= (uint32_t)K ? (float)miss / SAMPLES : 0.f,
                        std::log1p((float)sub[0]), std::log1p((float)sub[1]),
                        (float)sub[2] * 1000.f / (float)std::max(n, 1u), std::log1p((float)sub[3])};
    const float *w = m->h_w.data();
    float x[F], h1[H], h2[H];
    for (int i = 0; i < F; ++i) x[i] = (f[i] - m->norm.fmean[i]) / m->norm.fstd[i];
    for (int o = 0; o < H; ++o) {
        float a = w[OB1 + o];
        for (int i = 0; i < F; ++i) a += w[OW1 + o * F + i] * x[i];
        h1[o] = std::max(a, 0.f);
    }
    for (int o = 0; o < H; ++o) {
        float a = w[OB2 + o];
        for (int i = 0; i < H; ++i) a += w[OW2 + o * H + i] * h1[i];
        h2[o] = std::max(a, 0.f);
    }
    for (int o = 0; o < O; ++o) {
        float a = w[OB3 + o];
        for (int i = 0; i < H; ++i) a += w[OW3 + o * H + i] * h2[i];
        h_pred[o] = a * m->norm.tstd[o] + m->norm.tmean[o];
    }
    return GWFA_OK;
}

}  // extern "C"
