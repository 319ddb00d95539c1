// gwfa_noalloc.cu -- batch alignment that allocates no memory at all.
//
// Every other batch entry point of the library keeps its per-CTA hash slabs in
// memory it obtained with cudaMalloc (an engine).  Some callers cannot let a
// library allocate device memory: code running inside a custom device-memory
// allocator (calling back into an allocator there can deadlock or recurse),
// processes whose device memory has been reserved up front by another framework
// so that a new cudaMalloc fails or breaks its accounting, and latency-critical
// loops that cannot afford cudaMalloc's implicit device-wide synchronisation.
// For them, gwfa_align_noalloc runs the same alignment kernel with its scratch
// carved from one fixed, file-scope device array instead.
//
// That array is kNoallocScratchBytes (32 MiB) on every GPU that loads the
// library, for the life of the process.  It is shared by every call: each call
// re-initialises it (work-queue counter to zero, hash slabs to empty) before its
// kernel, so calls whose GPU work overlaps (two streams, or two host threads)
// race on it and must be serialised by the caller.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "gwfa_internal.cuh"

namespace {

constexpr uint64_t kNoallocScratchBytes = 32ull << 20;
constexpr uint64_t kHeadBytes = 256;   // the work-queue counter, then the slabs

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};   // context the address belongs to

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Identifier of the calling thread's current context (unique for the life of the
// process, so a device reset that replaces the primary context changes it); 0 if
// the driver cannot tell.  The driver functions are found through the runtime, so
// the library does not link the driver library itself.
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (CtxGetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (CtxGetIdFn)f;
        cudaGetLastError();
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of g_noalloc_scratch on the current device (the host-side name of
// the array is only a stand-in, not a device address).  Looked up once per device
// and context: the first call on a device does it, and again after a device reset
// has replaced the context the cached address belonged to.
int scratch_address(int dev, uint8_t **out) {
    if (dev < 0 || dev >= kMaxDevices) return GWFA_ERR_INVALID;
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return GWFA_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = ctx;
    }
    *out = (uint8_t *)g_scratch_addr[dev];
    return GWFA_OK;
}

}  // namespace

extern "C" int gwfa_align_noalloc(const gwfa_graph *g, uint32_t n_queries, const uint32_t *d_words,
                                  const uint64_t *d_q_off, const uint32_t *d_v_s,
                                  const uint32_t *d_v_e, const int32_t *d_status, uint32_t log2_tiles,
                                  const gwfa_opts *opts, gwfa_result *d_out, void *stream) {
    if (!g || !d_words || !d_q_off || !d_v_s || !d_v_e || !d_out) return GWFA_ERR_INVALID;
    const gwfa_opts o = opts ? *opts : gwfa_opts{0, 0, -1, 0};
    if (o.max_lag < 0 || o.traceback != 0 || o.ends != 0 || o.evict_lag != 0) return GWFA_ERR_INVALID;
    if (log2_tiles == 0) log2_tiles = 15;
    const bool prune = o.max_lag > 0;
    if (log2_tiles < 8 || log2_tiles > gwfa::kMaxLog2Tiles) return GWFA_ERR_INVALID;
    const uint64_t slab = gwfa::slab_layout(log2_tiles, prune).total;
    if (slab + kHeadBytes > kNoallocScratchBytes) return GWFA_ERR_CAPACITY;   // does not fit the array
    if (n_queries == 0) return GWFA_OK;
    if (cudaSetDevice(g->device) != cudaSuccess) return GWFA_ERR_CUDA;
    uint8_t *base = nullptr;
    int st = scratch_address(g->device, &base);
    if (st) return st;
    const uint32_t ctas = (uint32_t)((kNoallocScratchBytes - kHeadBytes) / slab);
    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's contents: reset what must start empty
    if (cudaMemsetAsync(base, 0, kHeadBytes, s) != cudaSuccess) return GWFA_ERR_CUDA;
    if (gwfa::launch_slab_init(base + kHeadBytes, slab, ctas, log2_tiles, prune, s) != cudaSuccess)
        return GWFA_ERR_CUDA;
    gwfa::TierArgs a{};
    a.g = g->dev();
    a.qwords = d_words;
    a.q_off = d_q_off;
    a.v_s = d_v_s;
    a.v_e = d_v_e;
    a.qstatus = d_status;   // a query the packing rejected keeps its status
    a.out = d_out;
    a.count_val = n_queries;
    a.head = (uint32_t *)base;
    a.slabs = base + kHeadBytes;
    a.slab_bytes = slab;
    a.log2cap = log2_tiles;
    a.max_lag = o.max_lag;
    a.max_score = o.max_score;
    return gwfa::launch_align(a, prune, ctas, 512, s) == cudaSuccess ? GWFA_OK : GWFA_ERR_CUDA;
}
