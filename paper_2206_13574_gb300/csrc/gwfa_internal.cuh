// gwfa_internal.cuh -- shared declarations of the CUDA library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/gwfa.h"

namespace gwfa {

// Host-side profiler range (NVTX): names a phase of a library call on the timeline
// of a profiler that is attached; a few nanoseconds when none is.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// A tile groups the 8 diagonals k = 8*kb .. 8*kb+7 of one vertex: its 8 offsets
// H~_{v,k} are one 32-byte sector (exact mode) and are processed by 8 adjacent
// lanes of a warp, so that the expand step (Alg. 3) is a shuffle inside the tile.
constexpr int kTile = 8;
constexpr uint64_t kEmptyKey = ~0ull;

// Packed graph resident on the device (a1): labels 2-bit packed, base t of a word
// in bits 2t..2t+1, every vertex starting on a word boundary, 2 zero pad words at
// the end so that a 32-base window may always read two consecutive words.
// vinfo[v] = {first word of the label, |v|, first out-arc, end of out-arcs}: one
// 16-byte load gives everything the extension of a diagonal of v needs.
struct DevGraph {
    const uint32_t *words;
    const uint4 *vinfo;
    const uint32_t *arc_dst;
    uint32_t nv;
};

// List entry: tile slot, vertex, tile index kb (diagonals 8kb .. 8kb+7).
struct __align__(16) LEnt {
    uint32_t slot;
    uint32_t v;
    int32_t kb;
    uint32_t pad;
};
// Extended-frontier header: slot | live-lane mask << 24, vertex, kb, |v|.
struct __align__(16) EHdr {
    uint32_t slot_mask;
    uint32_t v;
    int32_t kb;
    uint32_t lv;
};
constexpr uint32_t kMaxLog2Tiles = 24;   // slot must fit the 24 low bits of EHdr

// Hash slot of one tile, one 64-byte line in exact mode (128 in pruning mode):
// key (v << 32 | kb, all ones = empty), the two lane-mask words of the phase
// parities, and the 8 offsets; in pruning mode also the 8 trace indices (Alg. 5)
// of the diagonals, used with traceback.  A tile visit touches a single line.
template <class T>
struct alignas(sizeof(T) == 4 ? 64 : 128) SlotT {
    unsigned long long key;
    uint32_t reg[2];
    T vals[kTile];
    uint32_t trace[sizeof(T) == 4 ? 1 : kTile];
};
// Extended-frontier entry: header + snapshot of the 8 offsets (and, in pruning
// mode, of their trace indices) after extension.
template <class T>
struct alignas(sizeof(T) == 4 ? 64 : 128) EEntT {
    EHdr hdr;
    T vals[kTile];
    uint32_t trace[sizeof(T) == 4 ? 1 : kTile];
};

// Per-CTA slab layout (all arrays 256-byte aligned), cap = 2^log2 tiles.
struct SlabLayout {
    uint64_t slots, touched, qlist, slist0, slist1, elist, req, reqt, trace, total, slot_bytes;
};

__host__ __device__ inline uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

__host__ __device__ inline SlabLayout slab_layout(uint32_t log2cap, bool prune) {
    const uint64_t cap = 1ull << log2cap;
    const uint64_t sb = prune ? sizeof(SlotT<long long>) : sizeof(SlotT<int>);
    const uint64_t eb = prune ? sizeof(EEntT<long long>) : sizeof(EEntT<int>);
    SlabLayout L;
    uint64_t o = 0;
    L.slot_bytes = sb;
    L.slots = o;   o = align256(o + cap * sb);
    L.touched = o; o = align256(o + cap * 4);
    L.qlist = o;   o = align256(o + cap * sizeof(LEnt));
    L.slist0 = o;  o = align256(o + cap * sizeof(LEnt));
    L.slist1 = o;  o = align256(o + cap * sizeof(LEnt));
    L.elist = o;   o = align256(o + cap * eb);
    L.req = o;     o = align256(o + (prune ? cap * 16 : 0));
    L.reqt = o;    o = align256(o + (prune ? cap * 4 : 0));    // trace index of each spill request
    L.trace = o;   o = align256(o + (prune ? cap * 2 * 8 : 0));   // Alg. 5's T: (v, t) pairs
    L.total = o;
    return L;
}

// Arguments of one tier launch of the alignment kernel.
struct TierArgs {
    DevGraph g;
    const uint32_t *qwords;     // packed queries; query i starts at word (q_off[i] >> 4) + i
    const uint64_t *q_off;      // byte offsets of the ASCII queries, n + 1
    const uint32_t *v_s, *v_e;
    const int32_t *qstatus;     // optional pre-status (pack errors)
    gwfa_result *out;
    const uint32_t *list;       // query ids to run (NULL: identity)
    const uint32_t *list_count; // device count (NULL: use count_val)
    uint32_t count_val;
    uint32_t list_offset;       // queue position t runs list[list_offset + t]
    uint32_t *retry;            // overflowing query ids for the next tier (NULL: last tier)
    uint32_t *retry_count;
    uint32_t *head;             // work-queue head
    uint8_t *slabs;
    uint64_t slab_bytes;
    uint32_t log2cap;
    int32_t max_lag;
    int32_t max_score;
    unsigned long long *stats;  // optional, kStatWords per query id (see gwfa_engine_set_stats)
    int q_smem;                 // query words are in shared memory (server kernel)
    int traceback;              // 64-bit values carry a trace index (Alg. 5-6) instead of a base
    int ends;                   // formulation variant flags (GWFA_FREE_START / _FREE_END / _EXTEND)
    int evict_lag;              // memory bound on H~ (pruning mode): lag behind a_max, 0 = off
    int evict_every;            // scores between two evictions
    uint32_t *paths;            // traceback: path_cap vertex ids per query id
    uint32_t *path_len;         // traceback: walk length per query id (may exceed path_cap)
    uint32_t path_cap;
};
constexpr int kStatWords = 8;

// A serving request as the host publishes it (pinned, mapped host memory).
struct ReqDesc {
    unsigned long long ticket;
    uint32_t n, v_s, v_e, pad;
    uint64_t pad2;
};

// Arguments of the persistent server kernel; the rings live in mapped host memory.
struct ServerArgs {
    DevGraph g;
    uint8_t *slabs;
    uint64_t slab_bytes[2];
    uint64_t big_offset;           // byte offset of the class-1 slabs
    uint32_t log2cap[2];
    uint32_t n_small;              // CTAs serving class 0
    const ReqDesc *desc[2];
    const uint32_t *arena[2];      // packed query words, slot_words per ring slot
    gwfa_result *results[2];
    unsigned long long *done[2];   // ticket + 1 once results[slot] is final
    const unsigned long long *tail[2];
    unsigned long long *head;      // device, per class
    const unsigned long long *stop;
    unsigned long long *timeouts;  // device: CTAs that left after an idle period
    unsigned int *idle_votes;      // device: CTAs currently idle for wait_limit polls or more
    uint32_t n_ctas;
    uint32_t ring, slot_words;
    uint32_t wait_limit, sleep_ns;
    int32_t max_lag, max_score;
};

// launchers (gwfa_kernels.cu)
cudaError_t launch_align(const TierArgs &a, bool prune, uint32_t ctas, uint32_t threads,
                         cudaStream_t st);
cudaError_t launch_pack(uint32_t nq, const char *d_q, const uint64_t *d_off, uint32_t *d_words,
                        int32_t *d_status, cudaStream_t st);
cudaError_t launch_fill(void *p, uint64_t bytes, cudaStream_t st);
cudaError_t launch_slab_init(uint8_t *slabs, uint64_t slab_bytes, uint32_t n_slabs, uint32_t log2cap,
                             bool prune, cudaStream_t st);
int align_occupancy(bool prune, uint32_t threads, int *blocks_per_sm);
cudaError_t preload_kernels();
cudaError_t launch_server(const ServerArgs &a, bool prune, uint32_t ctas, uint32_t threads,
                          uint32_t smem_bytes, cudaStream_t st);

}  // namespace gwfa

struct gwfa_graph {
    int device = 0;
    uint32_t nv = 0;
    uint64_t na = 0, total = 0, n_words = 0;
    uint32_t max_outdeg = 0;
    int has_cycles = 0;
    std::vector<uint32_t> h_arc_off, h_arc_dst, h_vlen;
    uint32_t *d_words = nullptr, *d_arc_dst = nullptr;
    uint4 *d_vinfo = nullptr;
    uint64_t device_bytes = 0;
    // plain-path workspace (one slab), guarded by mu
    mutable std::mutex mu;
    mutable uint8_t *plain_slab = nullptr;
    mutable uint32_t plain_log2 = 0;
    mutable bool plain_prune = false;
    mutable uint8_t *plain_stage = nullptr;   // query bytes + words + counters + result
    mutable uint64_t plain_stage_bytes = 0;
    mutable cudaStream_t stream = nullptr;
    gwfa::DevGraph dev() const {
        return gwfa::DevGraph{d_words, d_vinfo, d_arc_dst, nv};
    }
};

struct gwfa_engine {
    const gwfa_graph *g = nullptr;
    gwfa_engine_config cfg{};
    uint8_t *slabs[GWFA_MAX_TIERS] = {};
    uint64_t slab_bytes[GWFA_MAX_TIERS] = {};
    uint8_t *wide_slabs = nullptr, *huge_slabs = nullptr;
    uint64_t wide_slab_bytes = 0, huge_slab_bytes = 0;
    cudaStream_t side = nullptr, side2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr;
    uint32_t *counters = nullptr;   // per tier: head, retry_count; plus retry lists
    uint32_t *retry_lists = nullptr;
    uint64_t retry_cap = 0;
    // staging for the host-buffer entry point
    uint8_t *stage = nullptr;
    uint64_t stage_bytes = 0;
    cudaStream_t stream = nullptr;
    uint64_t device_bytes = 0;
    uint32_t last_launches = 0;
    unsigned long long *stats = nullptr;
    uint32_t *paths = nullptr, *path_len = nullptr;
    uint32_t path_cap = 0;
    std::mutex mu;
};
