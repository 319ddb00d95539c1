// gwfa_server.cu -- serving: continuous batching over a resident graph.
//
// Requests are published into two rings in pinned, device-mapped host memory
// (class 0: ordinary queries on CTAs with small hash slabs; class 1: queries
// predicted to need a large hash).  A persistent kernel (server_kernel in
// gwfa_kernels.cu) takes them as its CTAs free up and writes each result plus a
// completion tag straight back to host memory, so requests that arrive while
// others are on the GPU start without waiting for a batch boundary.  Admission:
// a request is placed in the class its predicted hash memory fits (the learned
// cost model when one is attached, else its length); a request that overflows a
// small slab anyway is re-queued into class 1 by the host, transparently.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gwfa_internal.cuh"

extern "C" int gwfa_model_predict_host(const gwfa_model *m, const char *q, uint32_t n, uint32_t v_s,
                                       uint32_t v_e, float *h_pred);

namespace {

int sstat(cudaError_t e) {
    if (e == cudaSuccess) return GWFA_OK;
    return e == cudaErrorMemoryAllocation ? GWFA_ERR_OOM : GWFA_ERR_CUDA;
}

constexpr uint64_t kClassShift = 56;

}  // namespace

struct gwfa_server {
    const gwfa_graph *g = nullptr;
    const gwfa_model *model = nullptr;
    gwfa_server_config cfg{};
    gwfa_opts opts{};
    bool prune = false;
    uint8_t *slabs = nullptr;
    uint64_t slab_bytes[2] = {0, 0}, big_offset = 0;
    // one pinned, mapped host block: descriptors, arenas, results, done tags, tails, stop
    uint8_t *host = nullptr;
    uint64_t host_bytes = 0;
    gwfa::ReqDesc *desc[2] = {};
    uint32_t *arena[2] = {};
    gwfa_result *res[2] = {};
    unsigned long long *done[2] = {};
    unsigned long long *tail[2] = {};
    unsigned long long *stop = nullptr;
    unsigned long long *d_head = nullptr, *d_timeouts = nullptr;
    unsigned int *d_votes = nullptr;
    gwfa::ServerArgs args{};
    uint32_t slot_words = 0, smem_bytes = 0;
    cudaStream_t stream = nullptr;
    bool launched = false;
    std::mutex mu;
    uint64_t next[2] = {0, 0};
    std::vector<uint8_t> busy[2];
    std::unordered_map<uint64_t, uint64_t> redirect;   // user ticket -> ticket now in flight
    uint64_t n_submitted = 0, n_completed = 0, n_requeued = 0, n_launches = 0;
};

namespace {

template <class T> T *host_take(uint8_t *base, uint64_t &off, uint64_t bytes) {
    T *p = (T *)(base + off);
    off = gwfa::align256(off + bytes);
    return p;
}

int dev_ptr(void **d, void *h) { return sstat(cudaHostGetDevicePointer(d, h, 0)); }

// (Re)start the persistent kernel if it is not running (it leaves on idle timeout).
int ensure_running(gwfa_server *sv) {
    if (sv->launched) {
        const cudaError_t q = cudaStreamQuery(sv->stream);
        if (q == cudaErrorNotReady) return GWFA_OK;
        if (q != cudaSuccess) return sstat(q);
    }
    const uint32_t ctas = sv->cfg.ctas_small + sv->cfg.ctas_big;
    // a new generation of CTAs starts with no idle votes (stream-ordered after the last)
    int st = sstat(cudaMemsetAsync(sv->d_votes, 0, sizeof(unsigned int), sv->stream));
    if (!st) st = sstat(gwfa::launch_server(sv->args, sv->prune, ctas, sv->cfg.threads, sv->smem_bytes, sv->stream));
    if (!st) {
        sv->launched = true;
        sv->n_launches++;
    }
    return st;
}

// Publish one request (query already packed into `words`) into class `cls`.
int publish(gwfa_server *sv, int cls, const uint32_t *words, uint32_t n, uint32_t vs, uint32_t ve,
            uint64_t *ticket) {
    const uint64_t seq = sv->next[cls];
    const uint32_t slot = (uint32_t)(seq % sv->cfg.ring_slots);
    if (sv->busy[cls][slot]) return GWFA_PENDING;   // ring full: the caller retries later
    const uint32_t nw = (n + 15) >> 4;
    memcpy(sv->arena[cls] + (uint64_t)slot * sv->slot_words, words, (uint64_t)nw * 4);
    gwfa::ReqDesc &d = sv->desc[cls][slot];
    d.ticket = seq;
    d.n = n;
    d.v_s = vs;
    d.v_e = ve;
    sv->busy[cls][slot] = 1;
    sv->next[cls] = seq + 1;
    // the descriptor and words must be visible before the tail that publishes them
    std::atomic_thread_fence(std::memory_order_release);
    __atomic_store_n(sv->tail[cls], (unsigned long long)(seq + 1), __ATOMIC_RELEASE);
    *ticket = ((uint64_t)cls << kClassShift) | seq;
    return ensure_running(sv);
}

int pack_query(const char *q, uint32_t n, std::vector<uint32_t> &w) {
    w.assign(((n + 15) >> 4) + 1, 0u);
    for (uint32_t p = 0; p < n; ++p) {
        int c;
        switch (q[p]) {
        case 'A': case 'a': c = 0; break;
        case 'C': case 'c': c = 1; break;
        case 'G': case 'g': c = 2; break;
        case 'T': case 't': c = 3; break;
        default: return GWFA_ERR_INVALID;
        }
        w[p >> 4] |= (uint32_t)c << (2 * (p & 15));
    }
    return GWFA_OK;
}

}  // namespace

extern "C" {

int gwfa_server_default_config(const gwfa_graph *g, gwfa_server_config *c) {
    if (!g || !c) return GWFA_ERR_INVALID;
    memset(c, 0, sizeof(*c));
    int sms = 0;
    if (cudaSetDevice(g->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess)
        return GWFA_ERR_CUDA;
    // 512-thread CTAs, four per SM; half an SM's worth of them hold large slabs
    // (and serve small requests when no large one waits)
    c->threads = 512;
    c->ctas_big = (uint32_t)std::max(sms / 2, 1);
    c->ctas_small = (uint32_t)sms * 4 - c->ctas_big;
    c->log2_small = 17;
    c->log2_big = 21;
    c->ring_slots = 4096;
    c->max_query_len = 131072;
    c->idle_us = 200000;
    c->big_length = 40000;
    return GWFA_OK;
}

int gwfa_server_create(const gwfa_graph *g, const gwfa_server_config *cfg, const gwfa_opts *opts,
                       const gwfa_model *model, gwfa_server **out) {
    if (!g || !cfg || !out) return GWFA_ERR_INVALID;
    *out = nullptr;
    const gwfa_server_config &c = *cfg;
    if (c.ctas_small == 0 || c.threads % 32 || c.threads < 64 || c.threads > 512 || c.ring_slots == 0 ||
        c.max_query_len == 0 || c.log2_small < 8 || c.log2_small > gwfa::kMaxLog2Tiles ||
        (c.ctas_big && (c.log2_big < 8 || c.log2_big > gwfa::kMaxLog2Tiles)))
        return GWFA_ERR_INVALID;
    gwfa_opts o = opts ? *opts : gwfa_opts{0, 0, -1, 0};
    if (o.max_lag < 0 || o.traceback != 0 || o.ends != 0 || o.evict_lag != 0) return GWFA_ERR_INVALID;
    int st = sstat(cudaSetDevice(g->device));
    if (st) return st;
    gwfa_server *sv = new (std::nothrow) gwfa_server();
    if (!sv) return GWFA_ERR_OOM;
    sv->g = g;
    sv->model = model;
    sv->cfg = c;
    sv->opts = o;
    sv->prune = o.max_lag > 0;
    sv->slot_words = (c.max_query_len + 15) / 16 + 2;
    sv->smem_bytes = sv->slot_words * 4 + 16;
    sv->busy[0].assign(c.ring_slots, 0);
    sv->busy[1].assign(c.ring_slots, 0);
    // device slabs: class 0 then class 1
    sv->slab_bytes[0] = gwfa::slab_layout(c.log2_small, sv->prune).total;
    sv->slab_bytes[1] = c.ctas_big ? gwfa::slab_layout(c.log2_big, sv->prune).total : 0;
    sv->big_offset = sv->slab_bytes[0] * c.ctas_small;
    const uint64_t slab_total = sv->big_offset + sv->slab_bytes[1] * c.ctas_big;
    st = sstat(cudaMalloc(&sv->slabs, slab_total));
    if (!st) st = sstat(cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking));
    if (!st)
        st = sstat(gwfa::launch_slab_init(sv->slabs, sv->slab_bytes[0], c.ctas_small, c.log2_small, sv->prune,
                                          sv->stream));
    if (!st && c.ctas_big)
        st = sstat(gwfa::launch_slab_init(sv->slabs + sv->big_offset, sv->slab_bytes[1], c.ctas_big,
                                          c.log2_big, sv->prune, sv->stream));
    if (!st) st = sstat(cudaMalloc(&sv->d_head, 2 * sizeof(unsigned long long)));
    if (!st) st = sstat(cudaMalloc(&sv->d_timeouts, sizeof(unsigned long long)));
    if (!st) st = sstat(cudaMalloc(&sv->d_votes, sizeof(unsigned int)));
    if (!st) st = sstat(cudaMemsetAsync(sv->d_head, 0, 2 * sizeof(unsigned long long), sv->stream));
    if (!st) st = sstat(cudaMemsetAsync(sv->d_timeouts, 0, sizeof(unsigned long long), sv->stream));
    // pinned, mapped host block
    uint64_t off = 0;
    const uint64_t R = c.ring_slots;
    uint64_t offs[12];
    int k = 0;
    for (int cls = 0; cls < 2; ++cls) {
        offs[k++] = off; off = gwfa::align256(off + R * sizeof(gwfa::ReqDesc));
        offs[k++] = off; off = gwfa::align256(off + R * sv->slot_words * 4);
        offs[k++] = off; off = gwfa::align256(off + R * sizeof(gwfa_result));
        offs[k++] = off; off = gwfa::align256(off + R * 8);
        offs[k++] = off; off = gwfa::align256(off + 8);
    }
    offs[k++] = off; off = gwfa::align256(off + 8);
    sv->host_bytes = off;
    if (!st) st = sstat(cudaHostAlloc((void **)&sv->host, off, cudaHostAllocMapped | cudaHostAllocPortable));
    if (st) { gwfa_server_destroy(sv); return st; }
    memset(sv->host, 0, off);
    k = 0;
    for (int cls = 0; cls < 2; ++cls) {
        sv->desc[cls] = (gwfa::ReqDesc *)(sv->host + offs[k++]);
        sv->arena[cls] = (uint32_t *)(sv->host + offs[k++]);
        sv->res[cls] = (gwfa_result *)(sv->host + offs[k++]);
        sv->done[cls] = (unsigned long long *)(sv->host + offs[k++]);
        sv->tail[cls] = (unsigned long long *)(sv->host + offs[k++]);
    }
    sv->stop = (unsigned long long *)(sv->host + offs[k++]);
    gwfa::ServerArgs &a = sv->args;
    a.g = g->dev();
    a.slabs = sv->slabs;
    a.slab_bytes[0] = sv->slab_bytes[0];
    a.slab_bytes[1] = sv->slab_bytes[1];
    a.big_offset = sv->big_offset;
    a.log2cap[0] = c.log2_small;
    a.log2cap[1] = c.ctas_big ? c.log2_big : c.log2_small;
    a.n_small = c.ctas_small;
    for (int cls = 0; cls < 2 && !st; ++cls) {
        void *p;
        st = dev_ptr(&p, sv->desc[cls]);
        a.desc[cls] = (const gwfa::ReqDesc *)p;
        if (!st) st = dev_ptr(&p, sv->arena[cls]);
        a.arena[cls] = (const uint32_t *)p;
        if (!st) st = dev_ptr(&p, sv->res[cls]);
        a.results[cls] = (gwfa_result *)p;
        if (!st) st = dev_ptr(&p, sv->done[cls]);
        a.done[cls] = (unsigned long long *)p;
        if (!st) st = dev_ptr(&p, sv->tail[cls]);
        a.tail[cls] = (const unsigned long long *)p;
    }
    void *p = nullptr;
    if (!st) st = dev_ptr(&p, sv->stop);
    a.stop = (const unsigned long long *)p;
    a.head = sv->d_head;
    a.timeouts = sv->d_timeouts;
    a.idle_votes = sv->d_votes;
    a.n_ctas = c.ctas_small + c.ctas_big;
    a.ring = c.ring_slots;
    a.slot_words = sv->slot_words;
    a.sleep_ns = 2000;
    a.wait_limit = std::max<uint32_t>(c.idle_us / 2, 1);
    a.max_lag = o.max_lag;
    a.max_score = o.max_score;
    if (!st) st = sstat(cudaStreamSynchronize(sv->stream));
    if (st) { gwfa_server_destroy(sv); return st; }
    *out = sv;
    return GWFA_OK;
}

int gwfa_submit(gwfa_server *sv, const char *q, uint32_t n, uint32_t v_s, uint32_t v_e, uint64_t *ticket) {
    if (!sv || !ticket || (n && !q)) return GWFA_ERR_INVALID;
    if (n > sv->cfg.max_query_len || v_s >= sv->g->nv || v_e >= sv->g->nv) return GWFA_ERR_INVALID;
    std::vector<uint32_t> w;
    int st = pack_query(q, n, w);
    if (st) return st;
    // admission: the class whose hash slabs the predicted memory fits
    int cls = 0;
    if (sv->cfg.ctas_big) {
        if (sv->model) {
            float pred[GWFA_MODEL_TARGETS];
            if (gwfa_model_predict_host(sv->model, q, n, v_s, v_e, pred) == GWFA_OK) {
                const double tiles = std::expm1((double)pred[2]) * 0.25;   // diagonals -> tiles
                cls = tiles > 0.75 * (double)(1ull << sv->cfg.log2_small) ? 1 : 0;
            }
        } else {
            cls = n > sv->cfg.big_length ? 1 : 0;
        }
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (cudaSetDevice(sv->g->device) != cudaSuccess) return GWFA_ERR_CUDA;
    st = publish(sv, cls, w.data(), n, v_s, v_e, ticket);
    if (st == GWFA_OK) sv->n_submitted++;
    return st;
}

int gwfa_poll(gwfa_server *sv, uint64_t ticket, gwfa_result *out) {
    if (!sv || !out) return GWFA_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    uint64_t t = ticket;
    auto it = sv->redirect.find(ticket);
    if (it != sv->redirect.end()) t = it->second;
    const int cls = (int)(t >> kClassShift);
    const uint64_t seq = t & ((1ull << kClassShift) - 1);
    if (cls > 1 || seq >= sv->next[cls]) return GWFA_ERR_INVALID;
    const uint32_t slot = (uint32_t)(seq % sv->cfg.ring_slots);
    if (__atomic_load_n(sv->done[cls] + slot, __ATOMIC_ACQUIRE) != seq + 1) {
        if (cudaSetDevice(sv->g->device) != cudaSuccess) return GWFA_ERR_CUDA;
        const int st = ensure_running(sv);   // the kernel may have left on an idle timeout
        return st ? st : GWFA_PENDING;
    }
    gwfa_result r = sv->res[cls][slot];
    if (!sv->busy[cls][slot]) return GWFA_ERR_INVALID;   // collected already
    if (r.status == GWFA_ERR_CAPACITY && cls == 0 && sv->cfg.ctas_big) {
        // a misprediction: re-queue into the large-slab class from the same words
        const gwfa::ReqDesc d = sv->desc[0][slot];
        std::vector<uint32_t> w(sv->arena[0] + (uint64_t)slot * sv->slot_words,
                                sv->arena[0] + (uint64_t)slot * sv->slot_words + ((d.n + 15) >> 4) + 1);
        uint64_t nt;
        if (cudaSetDevice(sv->g->device) != cudaSuccess) return GWFA_ERR_CUDA;
        const int st = publish(sv, 1, w.data(), d.n, d.v_s, d.v_e, &nt);
        if (st == GWFA_PENDING) return GWFA_PENDING;   // class-1 ring full: keep the result, retry
        if (st) return st;
        sv->busy[0][slot] = 0;
        sv->redirect[ticket] = nt;
        sv->n_requeued++;
        return GWFA_PENDING;
    }
    sv->busy[cls][slot] = 0;
    if (it != sv->redirect.end()) sv->redirect.erase(it);
    sv->n_completed++;
    *out = r;
    return GWFA_OK;
}

int gwfa_poll_many(gwfa_server *sv, uint32_t n, const uint64_t *tickets, gwfa_result *out,
                   uint8_t *done_flags, uint32_t *n_done) {
    if (!sv || (n && (!tickets || !out || !done_flags)) || !n_done) return GWFA_ERR_INVALID;
    uint32_t k = 0;
    for (uint32_t i = 0; i < n; ++i) {
        if (done_flags[i]) continue;
        const int st = gwfa_poll(sv, tickets[i], out + i);
        if (st == GWFA_OK) {
            done_flags[i] = 1;
            ++k;
        } else if (st != GWFA_PENDING) {
            return st;
        }
    }
    *n_done = k;
    return GWFA_OK;
}

int gwfa_wait(gwfa_server *sv, uint64_t ticket, uint32_t timeout_ms, gwfa_result *out) {
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const int st = gwfa_poll(sv, ticket, out);
        if (st != GWFA_PENDING) return st;
        const auto el = std::chrono::steady_clock::now() - t0;
        if (std::chrono::duration_cast<std::chrono::milliseconds>(el).count() >= timeout_ms)
            return GWFA_ERR_TIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

int gwfa_server_get_stats(gwfa_server *sv, gwfa_server_stats *o) {
    if (!sv || !o) return GWFA_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    o->submitted = sv->n_submitted;
    o->completed = sv->n_completed;
    o->requeued = sv->n_requeued;
    o->launches = sv->n_launches;
    o->in_flight = sv->n_submitted - sv->n_completed;
    o->device_bytes = sv->big_offset + sv->slab_bytes[1] * sv->cfg.ctas_big;
    return GWFA_OK;
}

int gwfa_server_destroy(gwfa_server *sv) {
    if (!sv) return GWFA_ERR_INVALID;
    cudaSetDevice(sv->g->device);
    if (sv->stop) __atomic_store_n(sv->stop, 1ull, __ATOMIC_RELEASE);
    if (sv->stream) {
        cudaStreamSynchronize(sv->stream);   // CTAs see the stop flag within one poll
        cudaStreamDestroy(sv->stream);
    }
    cudaFree(sv->slabs);
    cudaFree(sv->d_head);
    cudaFree(sv->d_timeouts);
    cudaFree(sv->d_votes);
    if (sv->host) cudaFreeHost(sv->host);
    delete sv;
    return GWFA_OK;
}

}  // extern "C"
