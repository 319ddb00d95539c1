// gwfa_api.cu -- host side of the C ABI declared in include/gwfa.h.
//
// Graph upload (packing, arc merging, CSR), the plain one-query path, the
// engine (per-CTA slabs in tiers, retry lists) and the batch entry points.
// Every step of the alignment itself runs in the kernels of gwfa_kernels.cu.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "gwfa_internal.cuh"

using gwfa::TierArgs;

namespace {

int host_code(char c) {
    switch (c) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    default: return -1;
    }
}

template <class T>
int dmalloc(T **p, uint64_t bytes) {
    if (bytes == 0) bytes = 16;
    if (cudaMalloc((void **)p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return GWFA_ERR_OOM;
    }
    return GWFA_OK;
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return GWFA_OK;
    if (e == cudaErrorMemoryAllocation) return GWFA_ERR_OOM;
    return GWFA_ERR_CUDA;
}

// Grow-only device buffer.
int ensure(uint8_t **buf, uint64_t *have, uint64_t need) {
    if (*have >= need) return GWFA_OK;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    uint64_t want = std::max<uint64_t>(need, 1 << 20);
    if (dmalloc(buf, want)) return GWFA_ERR_OOM;
    *have = want;
    return GWFA_OK;
}

// Host reachability v_s -> v_e (Def. 2 assumes it; the paper's loop never ends otherwise).
bool reachable(const gwfa_graph *g, uint32_t vs, uint32_t ve) {
    if (vs == ve) return true;
    std::vector<uint8_t> seen(g->nv, 0);
    std::vector<uint32_t> st;
    st.push_back(vs);
    seen[vs] = 1;
    while (!st.empty()) {
        uint32_t v = st.back();
        st.pop_back();
        for (uint32_t a = g->h_arc_off[v]; a < g->h_arc_off[v + 1]; ++a) {
            uint32_t u = g->h_arc_dst[a];
            if (u == ve) return true;
            if (!seen[u]) { seen[u] = 1; st.push_back(u); }
        }
    }
    return false;
}

struct Carve {
    uint8_t *base;
    uint64_t off = 0;
    template <class T> T *take(uint64_t bytes) {
        T *p = (T *)(base + off);
        off = gwfa::align256(off + bytes);
        return p;
    }
};

uint64_t words_for(uint32_t nq, uint64_t nbases) { return (nbases >> 4) + nq + 2; }

}  // namespace

extern "C" {

const char *gwfa_strerror(int s) {
    switch (s) {
    case GWFA_OK: return "ok";
    case GWFA_PENDING: return "pending";
    case GWFA_ERR_INVALID: return "invalid argument";
    case GWFA_ERR_OOM: return "out of memory";
    case GWFA_ERR_CUDA: return "CUDA error";
    case GWFA_ERR_UNREACHABLE: return "end vertex not reachable from start vertex";
    case GWFA_ERR_EMPTY_FRONTIER: return "pruning emptied the wavefront";
    case GWFA_ERR_CAPACITY: return "workspace capacity exceeded";
    case GWFA_ERR_TIMEOUT: return "device wait timed out";
    case GWFA_ERR_SCORE_LIMIT: return "edit distance above max_score";
    case GWFA_ERR_NOT_RUN: return "query not run";
    default: return "unknown status";
    }
}

int gwfa_graph_create(uint32_t nv, const char *h_seq, const uint64_t *h_seq_off, uint64_t na,
                      const uint32_t *h_arc_src, const uint32_t *h_arc_dst, int device,
                      gwfa_graph **out) {
    gwfa::Range range_("gwfa_graph_create");
    if (!out || !h_seq_off || (nv > 0 && !h_seq) || (na > 0 && (!h_arc_src || !h_arc_dst)))
        return GWFA_ERR_INVALID;
    *out = nullptr;
    if (nv == 0 || nv >= 0x7FFFFFFFu) return GWFA_ERR_INVALID;
    // labels: non-empty, ACGT, 2-bit packed, each vertex on a word boundary
    std::vector<uint32_t> vstart(nv), vlen(nv);
    uint64_t nwords = 0, total = 0;
    for (uint32_t v = 0; v < nv; ++v) {
        if (h_seq_off[v + 1] <= h_seq_off[v]) return GWFA_ERR_INVALID;
        uint64_t L = h_seq_off[v + 1] - h_seq_off[v];
        if (L >= (1ull << 30)) return GWFA_ERR_INVALID;
        vlen[v] = (uint32_t)L;
        vstart[v] = (uint32_t)nwords;
        nwords += (L + 15) >> 4;
        total += L;
        if (nwords >= 0xFFFFFFF0ull) return GWFA_ERR_INVALID;
    }
    std::vector<uint32_t> words(nwords + 2, 0);
    for (uint32_t v = 0; v < nv; ++v) {
        const char *s = h_seq + h_seq_off[v];
        uint32_t *w = words.data() + vstart[v];
        for (uint32_t p = 0; p < vlen[v]; ++p) {
            int c = host_code(s[p]);
            if (c < 0) return GWFA_ERR_INVALID;
            w[p >> 4] |= (uint32_t)c << (2 * (p & 15));
        }
    }
    // arcs: validate, merge duplicates, CSR by source
    std::vector<std::pair<uint32_t, uint32_t>> arcs(na);
    int has_cycles = 0;
    for (uint64_t a = 0; a < na; ++a) {
        if (h_arc_src[a] >= nv || h_arc_dst[a] >= nv) return GWFA_ERR_INVALID;
        arcs[a] = {h_arc_src[a], h_arc_dst[a]};
        if (h_arc_dst[a] <= h_arc_src[a]) has_cycles = 1;
    }
    std::sort(arcs.begin(), arcs.end());
    arcs.erase(std::unique(arcs.begin(), arcs.end()), arcs.end());
    gwfa_graph *g = new (std::nothrow) gwfa_graph();
    if (!g) return GWFA_ERR_OOM;
    g->device = device;
    g->nv = nv;
    g->na = arcs.size();
    g->total = total;
    g->n_words = nwords + 2;
    g->has_cycles = has_cycles;
    g->h_arc_off.assign(nv + 1, 0);
    g->h_arc_dst.resize(arcs.size());
    for (auto &a : arcs) g->h_arc_off[a.first + 1]++;
    for (uint32_t v = 0; v < nv; ++v) {
        g->max_outdeg = std::max(g->max_outdeg, g->h_arc_off[v + 1]);
        g->h_arc_off[v + 1] += g->h_arc_off[v];
    }
    for (size_t a = 0; a < arcs.size(); ++a) g->h_arc_dst[a] = arcs[a].second;
    g->h_vlen = vlen;

    int st = cuda_status(cudaSetDevice(device));
    if (st) { delete g; return st; }
    std::vector<uint4> vinfo(nv);
    for (uint32_t v = 0; v < nv; ++v)
        vinfo[v] = make_uint4(vstart[v], vlen[v], g->h_arc_off[v], g->h_arc_off[v + 1]);
    st = dmalloc(&g->d_words, g->n_words * 4);
    if (!st) st = dmalloc(&g->d_vinfo, (uint64_t)nv * sizeof(uint4));
    if (!st) st = dmalloc(&g->d_arc_dst, std::max<uint64_t>(g->na, 1) * 4);
    if (!st) st = cuda_status(cudaMemcpy(g->d_words, words.data(), g->n_words * 4, cudaMemcpyHostToDevice));
    if (!st) st = cuda_status(cudaMemcpy(g->d_vinfo, vinfo.data(), (uint64_t)nv * sizeof(uint4), cudaMemcpyHostToDevice));
    if (!st && g->na) st = cuda_status(cudaMemcpy(g->d_arc_dst, g->h_arc_dst.data(), g->na * 4, cudaMemcpyHostToDevice));
    if (!st) st = cuda_status(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
    g->device_bytes = g->n_words * 4 + (uint64_t)nv * sizeof(uint4) + g->na * 4;
    if (st) { gwfa_graph_destroy(g); return st; }
    *out = g;
    return GWFA_OK;
}

int gwfa_graph_destroy(gwfa_graph *g) {
    if (!g) return GWFA_ERR_INVALID;
    cudaSetDevice(g->device);
    cudaFree(g->d_words);
    cudaFree(g->d_vinfo);
    cudaFree(g->d_arc_dst);
    cudaFree(g->plain_slab);
    cudaFree(g->plain_stage);
    if (g->stream) cudaStreamDestroy(g->stream);
    delete g;
    return GWFA_OK;
}

int gwfa_graph_get_info(const gwfa_graph *g, gwfa_graph_info *o) {
    if (!g || !o) return GWFA_ERR_INVALID;
    o->n_vertices = g->nv;
    o->max_out_degree = g->max_outdeg;
    o->n_arcs = g->na;
    o->total_bases = g->total;
    o->device_bytes = g->device_bytes;
    o->device = g->device;
    o->has_cycles = g->has_cycles;
    return GWFA_OK;
}

// ---------------------------------------------------------------- plain path

static int align_plain(const gwfa_graph *g, const char *h_q, uint32_t n, uint32_t vs, uint32_t ve,
                       const gwfa_opts &o, gwfa_result *out, uint32_t *h_path, uint32_t path_cap,
                       uint32_t *path_len);

// formulation variant flags: known bits only, and not combined with pruning; the
// memory bound on H~ needs pruning and the walk base in the payload (no traceback)
static bool ends_ok(const gwfa_opts &o) {
    return (o.ends & ~(GWFA_FREE_START | GWFA_FREE_END | GWFA_EXTEND)) == 0 && (o.ends == 0 || o.max_lag == 0) &&
           o.evict_lag >= 0 && o.evict_every >= 0 && (o.evict_lag == 0 || (o.max_lag > 0 && !o.traceback));
}

int gwfa_align(const gwfa_graph *g, const char *h_q, uint32_t n, uint32_t vs, uint32_t ve,
               const gwfa_opts *opts, gwfa_result *out) {
    gwfa_opts o = opts ? *opts : gwfa_opts{0, 0, -1, 0};
    if (o.traceback != 0) return GWFA_ERR_INVALID;   // the walk needs gwfa_align_path
    return align_plain(g, h_q, n, vs, ve, o, out, nullptr, 0, nullptr);
}

int gwfa_align_path(const gwfa_graph *g, const char *h_q, uint32_t n, uint32_t vs, uint32_t ve,
                    const gwfa_opts *opts, gwfa_result *out, uint32_t *h_path, uint32_t path_cap,
                    uint32_t *path_len) {
    gwfa_opts o = opts ? *opts : gwfa_opts{0, 0, -1, 0};
    if (!path_len || (path_cap && !h_path)) return GWFA_ERR_INVALID;
    o.traceback = 1;
    return align_plain(g, h_q, n, vs, ve, o, out, h_path, path_cap, path_len);
}

static int align_plain(const gwfa_graph *g, const char *h_q, uint32_t n, uint32_t vs, uint32_t ve,
                       const gwfa_opts &o, gwfa_result *out, uint32_t *h_path, uint32_t path_cap,
                       uint32_t *path_len) {
    gwfa::Range range_(o.traceback ? "gwfa_align_path" : "gwfa_align");
    if (!g || !out || (n > 0 && !h_q)) return GWFA_ERR_INVALID;
    memset(out, 0, sizeof(*out));
    out->edit_distance = -1;
    if (path_len) *path_len = 0;
    if (o.ends & GWFA_EXTEND) ve = vs;   // no end vertex
    if (vs >= g->nv || ve >= g->nv || o.max_lag < 0 || n >= 0x7FFFFFFFu || !ends_ok(o)) {
        out->status = GWFA_ERR_INVALID;
        return GWFA_ERR_INVALID;
    }
    if (!reachable(g, vs, ve)) {
        out->status = GWFA_ERR_UNREACHABLE;
        return GWFA_OK;
    }
    std::lock_guard<std::mutex> lk(g->mu);
    int st = cuda_status(cudaSetDevice(g->device));
    if (st) return st;
    const bool prune = o.max_lag > 0 || o.traceback;   // 64-bit values (walk base) and trace words
    // staging: query bytes | q_off[2] | v_s | v_e | words | status | head | result | path
    const uint64_t need = gwfa::align256(n + 16) + 256 * 6 + gwfa::align256(words_for(1, n) * 4) +
                          gwfa::align256(sizeof(gwfa_result)) + gwfa::align256((uint64_t)path_cap * 4) + 1024;
    st = ensure(&g->plain_stage, &g->plain_stage_bytes, need);
    if (st) return st;
    Carve c{g->plain_stage};
    char *d_q = c.take<char>(n + 16);
    uint64_t *d_off = c.take<uint64_t>(16);
    uint32_t *d_vs = c.take<uint32_t>(4);
    uint32_t *d_ve = c.take<uint32_t>(4);
    int32_t *d_status = c.take<int32_t>(4);
    uint32_t *d_head = c.take<uint32_t>(4);
    gwfa_result *d_res = c.take<gwfa_result>(sizeof(gwfa_result));
    uint32_t *d_words = c.take<uint32_t>(words_for(1, n) * 4);
    uint32_t *d_plen = c.take<uint32_t>(4);
    uint32_t *d_path = c.take<uint32_t>((uint64_t)path_cap * 4);
    uint64_t h_off[2] = {0, n};
    cudaStream_t s = g->stream;
    uint32_t log2 = g->plain_log2 && g->plain_prune == prune ? g->plain_log2 : (prune ? 15u : 16u);
    for (;;) {
        if (!g->plain_slab || g->plain_log2 != log2 || g->plain_prune != prune) {
            cudaFree(g->plain_slab);
            g->plain_slab = nullptr;
            const uint64_t bytes = gwfa::slab_layout(log2, prune).total;
            st = dmalloc(&g->plain_slab, bytes);
            if (st) return st;
            st = cuda_status(gwfa::launch_slab_init(g->plain_slab, bytes, 1, log2, prune, s));
            if (st) return st;
            g->plain_log2 = log2;
            g->plain_prune = prune;
        }
        if (n) cudaMemcpyAsync(d_q, h_q, n, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_off, h_off, 16, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_vs, &vs, 4, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_ve, &ve, 4, cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(d_head, 0, 4, s);
        st = cuda_status(gwfa::launch_pack(1, d_q, d_off, d_words, d_status, s));
        if (st) return st;
        TierArgs a{};
        a.g = g->dev();
        a.qwords = d_words;
        a.q_off = d_off;
        a.v_s = d_vs;
        a.v_e = d_ve;
        a.qstatus = d_status;
        a.out = d_res;
        a.list = nullptr;
        a.list_count = nullptr;
        a.count_val = 1;
        a.retry = nullptr;
        a.retry_count = nullptr;
        a.head = d_head;
        a.slabs = g->plain_slab;
        a.slab_bytes = gwfa::slab_layout(log2, prune).total;
        a.log2cap = log2;
        a.max_lag = o.max_lag;
        a.max_score = o.max_score;
        a.traceback = o.traceback ? 1 : 0;
        a.ends = o.ends;
        a.evict_lag = o.evict_lag;
        a.evict_every = o.evict_every ? o.evict_every : 64;
        a.paths = o.traceback ? d_path : nullptr;
        a.path_len = o.traceback ? d_plen : nullptr;
        a.path_cap = path_cap;
        if (o.traceback) cudaMemsetAsync(d_plen, 0, 4, s);
        st = cuda_status(gwfa::launch_align(a, prune, 1, 512, s));
        if (st) return st;
        st = cuda_status(cudaMemcpyAsync(out, d_res, sizeof(gwfa_result), cudaMemcpyDeviceToHost, s));
        if (!st && o.traceback) st = cuda_status(cudaMemcpyAsync(path_len, d_plen, 4, cudaMemcpyDeviceToHost, s));
        if (!st) st = cuda_status(cudaStreamSynchronize(s));
        if (!st && o.traceback && path_cap && *path_len)
            st = cuda_status(cudaMemcpy(h_path, d_path, (uint64_t)std::min(path_cap, *path_len) * 4,
                                        cudaMemcpyDeviceToHost));
        if (st) return st;
        if (out->status == GWFA_ERR_CAPACITY && log2 + 3 <= gwfa::kMaxLog2Tiles) {
            log2 += 3;   // grow the workspace and run again
            continue;
        }
        return GWFA_OK;
    }
}

// ---------------------------------------------------------------- engine

int gwfa_engine_default_config(const gwfa_graph *g, int prune, gwfa_engine_config *cfg) {
    if (!g || !cfg) return GWFA_ERR_INVALID;
    memset(cfg, 0, sizeof(*cfg));
    int st = cuda_status(cudaSetDevice(g->device));
    if (st) return st;
    int sms = 0, bps = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess)
        return GWFA_ERR_CUDA;
    // 512-thread CTAs, as many as fit on an SM (the kernel is bound by the latency
    // of dependent L2 round trips, so resident warps matter more than registers)
    cfg->threads = 512;
    if (gwfa::align_occupancy(prune != 0, cfg->threads, &bps) || bps < 1) bps = 1;
    cfg->wide = {0u, prune ? 18u : 19u, 512u, 0u};   // no concurrent classes by default
    cfg->huge = {0u, 22u, 512u, 0u};
    cfg->n_tiers = 3;
    cfg->tiers[0] = {(uint32_t)(sms * bps), prune ? 15u : 16u, 0u, 0u};
    cfg->tiers[1] = {(uint32_t)sms, 19u, 0u, 0u};
    cfg->tiers[2] = {(uint32_t)std::max(sms / 8, 1), 22u, 0u, 0u};
    cfg->prune_slabs = prune ? 1 : 0;
    cfg->max_queries = 1 << 16;
    cfg->max_bases = 1ull << 28;
    return GWFA_OK;
}

int gwfa_engine_destroy(gwfa_engine *e) {
    if (!e) return GWFA_ERR_INVALID;
    cudaSetDevice(e->g->device);
    for (int t = 0; t < GWFA_MAX_TIERS; ++t) cudaFree(e->slabs[t]);
    cudaFree(e->wide_slabs);
    cudaFree(e->huge_slabs);
    if (e->side) cudaStreamDestroy(e->side);
    if (e->side2) cudaStreamDestroy(e->side2);
    if (e->ev_join2) cudaEventDestroy(e->ev_join2);
    if (e->ev_fork) cudaEventDestroy(e->ev_fork);
    if (e->ev_join) cudaEventDestroy(e->ev_join);
    cudaFree(e->counters);
    cudaFree(e->retry_lists);
    cudaFree(e->stage);
    if (e->stream) cudaStreamDestroy(e->stream);
    delete e;
    return GWFA_OK;
}

static int engine_retry_capacity(gwfa_engine *e, uint64_t n) {
    if (e->retry_cap >= n) return GWFA_OK;
    cudaFree(e->retry_lists);
    e->retry_lists = nullptr;
    e->retry_cap = 0;
    uint64_t want = std::max<uint64_t>(n, 1024);
    if (dmalloc(&e->retry_lists, want * 4 * GWFA_MAX_TIERS)) return GWFA_ERR_OOM;
    e->retry_cap = want;
    return GWFA_OK;
}

int gwfa_engine_create(const gwfa_graph *g, const gwfa_engine_config *cfg, gwfa_engine **out) {
    gwfa::Range range_("gwfa_engine_create");
    if (!g || !cfg || !out) return GWFA_ERR_INVALID;
    *out = nullptr;
    if (cfg->n_tiers < 1 || cfg->n_tiers > GWFA_MAX_TIERS) return GWFA_ERR_INVALID;
    const uint32_t threads = cfg->threads ? cfg->threads : 128;
    if (threads % 32 || threads < 32 || threads > 1024) return GWFA_ERR_INVALID;
    for (uint32_t t = 0; t < cfg->n_tiers + 2; ++t) {
        const gwfa_tier &tt = t < cfg->n_tiers ? cfg->tiers[t] : (t == cfg->n_tiers ? cfg->wide : cfg->huge);
        if (t >= cfg->n_tiers && tt.ctas == 0) continue;   // class not used
        const uint32_t th = tt.threads;
        if (tt.ctas == 0 || tt.log2_tiles < 8 || tt.log2_tiles > gwfa::kMaxLog2Tiles ||
            (th && (th % 32 || th < 32 || th > 1024)))
            return GWFA_ERR_INVALID;
    }
    int st = cuda_status(cudaSetDevice(g->device));
    if (!st) st = cuda_status(gwfa::preload_kernels());
    if (st) return st;
    gwfa_engine *e = new (std::nothrow) gwfa_engine();
    if (!e) return GWFA_ERR_OOM;
    e->g = g;
    e->cfg = *cfg;
    e->cfg.threads = threads;
    st = cuda_status(cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking));
    for (uint32_t t = 0; !st && t < cfg->n_tiers; ++t) {
        e->slab_bytes[t] = gwfa::slab_layout(cfg->tiers[t].log2_tiles, cfg->prune_slabs != 0).total;
        const uint64_t bytes = e->slab_bytes[t] * cfg->tiers[t].ctas;
        st = dmalloc(&e->slabs[t], bytes);
        if (!st)
            st = cuda_status(gwfa::launch_slab_init(e->slabs[t], e->slab_bytes[t], cfg->tiers[t].ctas,
                                                    cfg->tiers[t].log2_tiles, cfg->prune_slabs != 0,
                                                    e->stream));
        e->device_bytes += bytes;
    }
    if (!st && cfg->huge.ctas) {
        e->huge_slab_bytes = gwfa::slab_layout(cfg->huge.log2_tiles, cfg->prune_slabs != 0).total;
        const uint64_t bytes = e->huge_slab_bytes * cfg->huge.ctas;
        st = dmalloc(&e->huge_slabs, bytes);
        if (!st)
            st = cuda_status(gwfa::launch_slab_init(e->huge_slabs, e->huge_slab_bytes, cfg->huge.ctas,
                                                    cfg->huge.log2_tiles, cfg->prune_slabs != 0,
                                                    e->stream));
        e->device_bytes += bytes;
    }
    if (!st) st = cuda_status(cudaStreamCreateWithFlags(&e->side2, cudaStreamNonBlocking));
    if (!st) st = cuda_status(cudaEventCreateWithFlags(&e->ev_join2, cudaEventDisableTiming));
    if (!st && cfg->wide.ctas) {
        e->wide_slab_bytes = gwfa::slab_layout(cfg->wide.log2_tiles, cfg->prune_slabs != 0).total;
        const uint64_t bytes = e->wide_slab_bytes * cfg->wide.ctas;
        st = dmalloc(&e->wide_slabs, bytes);
        if (!st)
            st = cuda_status(gwfa::launch_slab_init(e->wide_slabs, e->wide_slab_bytes, cfg->wide.ctas,
                                                    cfg->wide.log2_tiles, cfg->prune_slabs != 0,
                                                    e->stream));
        e->device_bytes += bytes;
    }
    if (!st) st = cuda_status(cudaStreamCreateWithFlags(&e->side, cudaStreamNonBlocking));
    if (!st) st = cuda_status(cudaEventCreateWithFlags(&e->ev_fork, cudaEventDisableTiming));
    if (!st) st = cuda_status(cudaEventCreateWithFlags(&e->ev_join, cudaEventDisableTiming));
    if (!st) st = dmalloc(&e->counters, 256);
    if (!st) st = engine_retry_capacity(e, cfg->max_queries);
    if (!st) st = cuda_status(cudaStreamSynchronize(e->stream));
    if (st) { gwfa_engine_destroy(e); return st; }
    *out = e;
    return GWFA_OK;
}

uint64_t gwfa_engine_device_bytes(const gwfa_engine *e) {
    return e ? e->device_bytes + e->retry_cap * 4 * GWFA_MAX_TIERS + e->stage_bytes : 0;
}

uint32_t gwfa_engine_last_launches(const gwfa_engine *e) { return e ? e->last_launches : 0; }

int gwfa_engine_last_retries(gwfa_engine *e, uint32_t *out) {
    if (!e || !out) return GWFA_ERR_INVALID;
    std::lock_guard<std::mutex> lk(e->mu);
    int st = cuda_status(cudaSetDevice(e->g->device));
    if (!st) st = cuda_status(cudaDeviceSynchronize());
    if (!st)
        st = cuda_status(cudaMemcpy(out, e->counters + GWFA_MAX_TIERS, GWFA_MAX_TIERS * 4,
                                    cudaMemcpyDeviceToHost));
    return st;
}

int gwfa_plan_schedule(uint32_t n, const float *h_pred, uint64_t tier0_tiles, uint64_t wide_tiles,
                       uint32_t *h_order, gwfa_schedule *out) {
    if ((n && (!h_pred || !h_order)) || !out) return GWFA_ERR_INVALID;
    std::vector<uint32_t> huge, big, small;
    // diagonals -> hash tiles: on the benchmark graphs a claimed 8-diagonal tile
    // holds about 6 visited diagonals; 0.25 tiles per diagonal leaves a margin of 1.5
    const double tile_per_diag = 0.25;
    for (uint32_t i = 0; i < n; ++i) {
        const double tiles = std::expm1((double)h_pred[(uint64_t)i * 4 + 2]) * tile_per_diag;
        if (wide_tiles && tiles > (double)wide_tiles) huge.push_back(i);
        else if (tiles > (double)tier0_tiles) big.push_back(i);
        else small.push_back(i);
    }
    auto by_cells = [&](uint32_t a, uint32_t b) {
        const float ca = h_pred[(uint64_t)a * 4 + 3], cb = h_pred[(uint64_t)b * 4 + 3];
        return ca != cb ? ca > cb : a < b;
    };
    std::sort(huge.begin(), huge.end(), by_cells);
    std::sort(big.begin(), big.end(), by_cells);
    std::sort(small.begin(), small.end(), by_cells);
    uint32_t k = 0;
    for (uint32_t i : huge) h_order[k++] = i;
    for (uint32_t i : big) h_order[k++] = i;
    for (uint32_t i : small) h_order[k++] = i;
    out->n_huge = (uint32_t)huge.size();
    out->n_wide = (uint32_t)big.size();
    return GWFA_OK;
}

int gwfa_engine_set_paths(gwfa_engine *e, uint32_t *d_paths, uint32_t path_cap, uint32_t *d_path_len) {
    if (!e || (path_cap && !d_paths)) return GWFA_ERR_INVALID;
    std::lock_guard<std::mutex> lk(e->mu);
    e->paths = d_paths;
    e->path_cap = path_cap;
    e->path_len = d_path_len;
    return GWFA_OK;
}

int gwfa_engine_set_stats(gwfa_engine *e, uint64_t *d_stats) {
    if (!e) return GWFA_ERR_INVALID;
    std::lock_guard<std::mutex> lk(e->mu);
    e->stats = (unsigned long long *)d_stats;
    return GWFA_OK;
}

int gwfa_pack_queries_device(uint32_t n_queries, const char *d_q, const uint64_t *d_q_off,
                             uint32_t *d_words, int32_t *d_status, void *stream) {
    if (!d_q_off || !d_words || (n_queries && !d_q)) return GWFA_ERR_INVALID;
    return cuda_status(gwfa::launch_pack(n_queries, d_q, d_q_off, d_words, d_status,
                                         (cudaStream_t)stream));
}

// Arguments of one alignment launch over queue positions [offset, offset + count)
// of `list` (or of the retry list given by list_count).
static TierArgs tier_args(gwfa_engine *e, const uint32_t *d_words, const uint64_t *d_q_off,
                          const uint32_t *d_vs, const uint32_t *d_ve, const int32_t *d_status,
                          const gwfa_opts &o, gwfa_result *d_out) {
    TierArgs a{};
    a.g = e->g->dev();
    a.qwords = d_words;
    a.q_off = d_q_off;
    a.v_s = d_vs;
    a.v_e = d_ve;
    a.qstatus = d_status;
    a.out = d_out;
    a.max_lag = o.max_lag;
    a.max_score = o.max_score;
    a.stats = e->stats;
    a.traceback = o.traceback ? 1 : 0;
    a.ends = o.ends;
    a.evict_lag = o.evict_lag;
    a.evict_every = o.evict_every ? o.evict_every : 64;
    a.paths = e->paths;
    a.path_len = e->path_len;
    a.path_cap = e->path_cap;
    return a;
}

static int run_tiers(gwfa_engine *e, uint32_t n, const uint32_t *d_words, const uint64_t *d_q_off,
                     const uint32_t *d_vs, const uint32_t *d_ve, const uint32_t *d_order,
                     const gwfa_schedule *sched, const int32_t *d_status, const gwfa_opts &o,
                     gwfa_result *d_out, cudaStream_t s) {
    int st = engine_retry_capacity(e, n);
    if (st) return st;
    const uint32_t T = e->cfg.n_tiers;
    uint32_t *heads = e->counters, *rcount = e->counters + GWFA_MAX_TIERS;
    st = cuda_status(cudaMemsetAsync(e->counters, 0, 256, s));
    if (st) return st;
    const bool prune = o.max_lag > 0 || o.traceback;   // 64-bit values
    e->last_launches = 0;
    // queue order: [huge | wide | tier 0]; the two first classes run on their own
    // CTAs, concurrently with tier 0, and hand their overflows to the retry tiers
    uint32_t n_huge = sched && e->huge_slabs ? std::min(sched->n_huge, n) : 0;
    uint32_t n_wide = sched && e->wide_slabs ? std::min(sched->n_wide, n - n_huge) : 0;
    struct Cls {
        const gwfa_tier *tier;
        uint8_t *slabs;
        uint64_t slab_bytes;
        cudaStream_t side;
        cudaEvent_t join;
        uint32_t count, offset, *head, *retry, *retry_count;
    } cls[2] = {
        {&e->cfg.huge, e->huge_slabs, e->huge_slab_bytes, e->side2, e->ev_join2, n_huge, 0,
         e->counters + 2 * GWFA_MAX_TIERS + 1, T > 1 ? e->retry_lists + (uint64_t)(T - 2) * e->retry_cap : nullptr,
         rcount + (T > 1 ? T - 2 : 0)},
        {&e->cfg.wide, e->wide_slabs, e->wide_slab_bytes, e->side, e->ev_join, n_wide, n_huge,
         e->counters + 2 * GWFA_MAX_TIERS, T > 1 ? e->retry_lists : nullptr, rcount},
    };
    // the classes' CTAs and tier 0's must be resident together (tier 0 would
    // otherwise fill every SM slot and the heaviest queries would start only after
    // it): tier 0 gives up the room of the class CTAs it runs beside
    const uint32_t t0_threads = e->cfg.tiers[0].threads ? e->cfg.tiers[0].threads : e->cfg.threads;
    uint64_t yield_threads = 0;
    uint32_t cctas[2] = {0, 0};
    for (int c = 0; c < 2; ++c) {
        if (!cls[c].count) continue;
        const uint32_t th = cls[c].tier->threads ? cls[c].tier->threads : e->cfg.threads;
        cctas[c] = std::min(cls[c].tier->ctas, cls[c].count);
        yield_threads += (uint64_t)cctas[c] * th;
    }
    const uint32_t t0_yield = (uint32_t)((yield_threads + t0_threads - 1) / t0_threads);
    const uint32_t t0_ctas = e->cfg.tiers[0].ctas > t0_yield ? e->cfg.tiers[0].ctas - t0_yield : 1;
    bool forked = false;
    for (int c = 0; c < 2; ++c) {
        if (!cls[c].count) continue;
        if (!forked) {
            st = cuda_status(cudaEventRecord(e->ev_fork, s));
            if (st) return st;
            forked = true;
        }
        TierArgs a = tier_args(e, d_words, d_q_off, d_vs, d_ve, d_status, o, d_out);
        a.list = d_order;
        a.count_val = cls[c].count;
        a.list_offset = cls[c].offset;
        a.retry = cls[c].retry;
        a.retry_count = cls[c].retry_count;
        a.head = cls[c].head;
        a.slabs = cls[c].slabs;
        a.slab_bytes = cls[c].slab_bytes;
        a.log2cap = cls[c].tier->log2_tiles;
        const uint32_t th = cls[c].tier->threads ? cls[c].tier->threads : e->cfg.threads;
        st = cuda_status(cudaStreamWaitEvent(cls[c].side, e->ev_fork, 0));
        if (!st) st = cuda_status(gwfa::launch_align(a, prune, cctas[c], th, cls[c].side));
        if (!st) st = cuda_status(cudaEventRecord(cls[c].join, cls[c].side));
        if (st) return st;
        e->last_launches++;
    }
    auto join_classes = [&]() -> int {
        for (int c = 0; c < 2; ++c)
            if (cls[c].count) {
                const int r = cuda_status(cudaStreamWaitEvent(s, cls[c].join, 0));
                if (r) return r;
            }
        return GWFA_OK;
    };
    for (uint32_t t = 0; t < T; ++t) {
        if (t == 1) {
            st = join_classes();   // the retry tiers also take the classes' overflows
            if (st) return st;
        }
        TierArgs a = tier_args(e, d_words, d_q_off, d_vs, d_ve, d_status, o, d_out);
        a.list = t == 0 ? d_order : e->retry_lists + (uint64_t)(t - 1) * e->retry_cap;
        a.list_count = t == 0 ? nullptr : rcount + (t - 1);
        a.count_val = t == 0 ? n - n_huge - n_wide : n;
        a.list_offset = t == 0 ? n_huge + n_wide : 0;
        a.retry = t + 1 < T ? e->retry_lists + (uint64_t)t * e->retry_cap : nullptr;
        a.retry_count = rcount + t;
        a.head = heads + t;
        a.slabs = e->slabs[t];
        a.slab_bytes = e->slab_bytes[t];
        a.log2cap = e->cfg.tiers[t].log2_tiles;
        const uint32_t th = e->cfg.tiers[t].threads ? e->cfg.tiers[t].threads : e->cfg.threads;
        st = cuda_status(gwfa::launch_align(a, prune, t == 0 ? t0_ctas : e->cfg.tiers[t].ctas, th, s));
        if (st) return st;
        e->last_launches++;
    }
    if (T == 1) return join_classes();
    return GWFA_OK;
}

int gwfa_align_batch_device(gwfa_engine *e, uint32_t n, const uint32_t *d_words,
                            const uint64_t *d_q_off, const uint32_t *d_vs, const uint32_t *d_ve,
                            const uint32_t *d_order, const gwfa_schedule *sched, const int32_t *d_status,
                            const gwfa_opts *opts, gwfa_result *d_out, void *stream) {
    gwfa::Range range_("gwfa_align_batch_device");
    if (!e || !d_words || !d_q_off || !d_vs || !d_ve || !d_out) return GWFA_ERR_INVALID;
    gwfa_opts o = opts ? *opts : gwfa_opts{0, 0, -1, 0};
    if (o.max_lag < 0 || !ends_ok(o)) return GWFA_ERR_INVALID;
    if ((o.max_lag > 0 || o.traceback) && !e->cfg.prune_slabs) return GWFA_ERR_INVALID;
    if (n == 0) return GWFA_OK;
    std::lock_guard<std::mutex> lk(e->mu);
    int st = cuda_status(cudaSetDevice(e->g->device));
    if (st) return st;
    // exactly the caller's stream (NULL = the legacy default stream), so the batch is
    // ordered after whatever produced its inputs on that stream
    return run_tiers(e, n, d_words, d_q_off, d_vs, d_ve, d_order, sched, d_status, o, d_out,
                     (cudaStream_t)stream);
}

int gwfa_align_batch(gwfa_engine *e, uint32_t n, const char *h_q, const uint64_t *h_q_off,
                     const uint32_t *h_vs, const uint32_t *h_ve, const uint32_t *h_order,
                     const gwfa_schedule *sched, const gwfa_opts *opts, gwfa_result *h_out, void *stream) {
    if (!e || !h_q_off || !h_vs || !h_ve || !h_out) return GWFA_ERR_INVALID;
    gwfa::Range range_("gwfa_align_batch");
    gwfa_opts o = opts ? *opts : gwfa_opts{0, 0, -1, 0};
    if (o.max_lag < 0 || !ends_ok(o)) return GWFA_ERR_INVALID;
    if ((o.max_lag > 0 || o.traceback) && !e->cfg.prune_slabs) return GWFA_ERR_INVALID;
    if (n == 0) return GWFA_OK;
    if (h_q_off[0] != 0) return GWFA_ERR_INVALID;
    const uint64_t nb = h_q_off[n];
    if (nb > 0 && !h_q) return GWFA_ERR_INVALID;
    std::lock_guard<std::mutex> lk(e->mu);
    int st = cuda_status(cudaSetDevice(e->g->device));
    if (st) return st;
    cudaStream_t s = stream ? (cudaStream_t)stream : e->stream;
    const uint64_t need = gwfa::align256(nb + 16) + gwfa::align256((uint64_t)(n + 1) * 8) +
                          3 * gwfa::align256((uint64_t)n * 4) + gwfa::align256((uint64_t)n * 4) +
                          gwfa::align256(words_for(n, nb) * 4) +
                          gwfa::align256((uint64_t)n * sizeof(gwfa_result)) + 4096;
    st = ensure(&e->stage, &e->stage_bytes, need);
    if (st) return st;
    Carve c{e->stage};
    char *d_q = c.take<char>(nb + 16);
    uint64_t *d_off = c.take<uint64_t>((uint64_t)(n + 1) * 8);
    uint32_t *d_vs = c.take<uint32_t>((uint64_t)n * 4);
    uint32_t *d_ve = c.take<uint32_t>((uint64_t)n * 4);
    uint32_t *d_order = c.take<uint32_t>((uint64_t)n * 4);
    int32_t *d_status = c.take<int32_t>((uint64_t)n * 4);
    uint32_t *d_words = c.take<uint32_t>(words_for(n, nb) * 4);
    gwfa_result *d_out = c.take<gwfa_result>((uint64_t)n * sizeof(gwfa_result));
    nvtxRangePushA("copy in + pack");
    st = cuda_status(cudaMemcpyAsync(d_q, h_q, nb, cudaMemcpyHostToDevice, s));
    if (!st) st = cuda_status(cudaMemcpyAsync(d_off, h_q_off, (uint64_t)(n + 1) * 8, cudaMemcpyHostToDevice, s));
    if (!st) st = cuda_status(cudaMemcpyAsync(d_vs, h_vs, (uint64_t)n * 4, cudaMemcpyHostToDevice, s));
    if (!st) st = cuda_status(cudaMemcpyAsync(d_ve, h_ve, (uint64_t)n * 4, cudaMemcpyHostToDevice, s));
    if (!st && h_order) st = cuda_status(cudaMemcpyAsync(d_order, h_order, (uint64_t)n * 4, cudaMemcpyHostToDevice, s));
    if (!st) st = cuda_status(gwfa::launch_pack(n, d_q, d_off, d_words, d_status, s));
    nvtxRangePop();
    nvtxRangePushA("alignment tiers");
    if (!st)
        st = run_tiers(e, n, d_words, d_off, d_vs, d_ve, h_order ? d_order : nullptr, sched, d_status, o,
                       d_out, s);
    nvtxRangePop();
    if (!st) e->last_launches += 1;
    nvtxRangePushA("copy out + wait");
    if (!st) st = cuda_status(cudaMemcpyAsync(h_out, d_out, (uint64_t)n * sizeof(gwfa_result), cudaMemcpyDeviceToHost, s));
    if (!st) st = cuda_status(cudaStreamSynchronize(s));
    nvtxRangePop();
    return st;
}

}  // extern "C"
