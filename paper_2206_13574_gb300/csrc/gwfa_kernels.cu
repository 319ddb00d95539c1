// gwfa_kernels.cu -- the graph wavefront alignment score loop on the GPU.
//
// One CTA runs the whole score loop of one query (Alg. 1): GwfExtend (Alg. 2,
// with the arc spills of Eq. 2's last case), the end test, GwfPrune (Alg. 4) and
// GwfExpand (Alg. 3), until the end cell (|q|, v_e, |v_e|) is on the wavefront.
// A persistent grid of CTAs pulls query ids from an atomic counter.
//
// Data layout (per CTA slab, reused across queries, see SlabLayout):
//   H~     open-addressing hash of tiles: key (v << 32 | kb) -> 8 offsets of the
//          diagonals k = 8 kb .. 8 kb + 7 of vertex v.  An offset is the int32 j
//          (exact mode) or the int64 (j << 32 | tag << 30 | base) (pruning mode,
//          base = spelled walk length before v, so W~ = base + j); absent = -1.
//          Entries persist for the whole query (an entry blocks re-spilling,
//          Alg. 2) and are wiped through the `touched` list when it ends.
//   reg    two lane-mask words per tile, one per phase parity.  A phase that
//          makes lanes live ORs their bits into its parity; the lane that finds
//          the word 0 appends the tile to that phase's list; the next phase takes
//          the mask with an exchange to 0, so each list holds every tile once.
//   Q      qlist: tiles live after GwfExpand (the queue Q of Alg. 1-3).
//   spill  slist[2]: tiles that received offset 0 by a spill and still have to
//          be extended in this score (Alg. 2 pushes them onto the queue being
//          drained).  Exact mode extends a won spill depth-first in the thread
//          that won it and only overflows to these lists; pruning mode goes
//          breadth first (see extend_round_prune).
//   E      the extended frontier (Q' of Alg. 2): header (slot, mask, v, kb, |v|)
//          and a snapshot of the 8 offsets after extension.  GwfExpand reads the
//          snapshot, so its sources are the offsets before any of its own writes
//          (the H~ / H~' split of Alg. 3) and it max-merges straight into H~.
//
// Order independence (why parallel execution gives the paper's exact result and
// work counts): in Alg. 2 every diagonal of the closure is extended exactly once
// from its starting offset, and a spill only fills an absent diagonal; in Alg. 3
// a diagonal enters Q' iff the max of its candidates beats its old offset, and
// its new value is that max.  Both are independent of the queue order.  Ties of
// the walk base (pruning mode only) are broken by the largest base within one
// breadth-first round of spills, which is what the oracle does too.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gwfa_internal.cuh"

namespace gwfa {

namespace {

constexpr long long kTagPend = 0, kTagFresh = 1, kTagSettled = 2;
constexpr uint32_t kBaseMask = 0x3FFFFFFFu;
constexpr int kStack = 6;   // depth-first spill stack per thread (exact mode)
// Tiles an 8-lane group takes per claim (both phases).  With a warp's four groups
// claiming together, one is fastest: two in flight hid more latency only while each
// group claimed alone, and their registers spill.
constexpr int kGroupTiles = 1;
constexpr uint32_t kNoTrace = 0x3FFFFFFFu;   // trace index of the start diagonal (no predecessor)

template <bool P> struct VT;
template <> struct VT<false> { using T = int; };
template <> struct VT<true> { using T = long long; };

__device__ __forceinline__ long long pk(int j, long long tag, uint32_t base) {
    return ((long long)j << 32) | (tag << 30) | (long long)base;
}
__device__ __forceinline__ int pj(long long v) { return (int)(v >> 32); }
__device__ __forceinline__ int pj(int v) { return v; }
__device__ __forceinline__ uint32_t pbase(long long v) { return (uint32_t)(v & kBaseMask); }
__device__ __forceinline__ uint32_t pbase(int) { return 0; }

template <bool P> struct Slab {
    using T = typename VT<P>::T;
    SlotT<T> *slots;
    uint32_t *touched;
    LEnt *qlist, *slist[2];
    EEntT<T> *elist;
    int4 *req;
    uint32_t *reqt;
    uint2 *trace;
    uint32_t cap, mask;
};

template <bool P>
__device__ __forceinline__ Slab<P> carve(uint8_t *base, uint32_t log2cap) {
    SlabLayout L = slab_layout(log2cap, P);
    Slab<P> s;
    s.slots = (SlotT<typename VT<P>::T> *)(base + L.slots);
    s.touched = (uint32_t *)(base + L.touched);
    s.qlist = (LEnt *)(base + L.qlist);
    s.slist[0] = (LEnt *)(base + L.slist0);
    s.slist[1] = (LEnt *)(base + L.slist1);
    s.elist = (EEntT<typename VT<P>::T> *)(base + L.elist);
    s.req = (int4 *)(base + L.req);
    s.reqt = (uint32_t *)(base + L.reqt);
    s.trace = (uint2 *)(base + L.trace);
    s.cap = 1u << log2cap;
    s.mask = s.cap - 1;
    return s;
}

// CTA-shared state of the query being aligned.
struct Sh {
    uint32_t qid;
    int err;
    int found;
    uint32_t nq[2];     // Q list length, by parity of the score that consumes it
    uint32_t ns[3];     // spill list length, rotating over three rounds (see align_one)
    uint32_t nreq[2];   // pending spill requests (pruning mode), by round parity
    uint32_t ne;        // extended-frontier entries this score
    uint32_t nt;        // tiles claimed (touched) this query
    uint32_t score_cells;
    // 32-bit shares of the 64-bit totals, folded in by thread 0 with an exchange
    // (a 64-bit shared-memory atomic costs far more than a 32-bit one)
    uint32_t spills32, visited32, pruned32;
    unsigned long long amax;
    unsigned long long cells, visited, pruned, spills, evicted;
    uint32_t nsurv;     // memory bound: tiles kept by the last eviction
    uint32_t peak;
    uint32_t claim[3];  // work counters of the phases, rotating (see align_one)
    uint32_t tlen;      // traceback: entries of T
    unsigned long long end_vp;   // traceback: vertex << 32 | trace of a diagonal at the end point
    unsigned long long t_start;  // query start (global timer, ns)
    unsigned long long t_phase;  // statistics: start of the current phase
    unsigned long long st[6];    // statistics: extend ns, expand ns, rounds, extended tiles,
                                 // expanded tiles, largest extended frontier (thread 0 only)
};

__device__ __forceinline__ void set_err(Sh &sh, int code) { atomicCAS(&sh.err, 0, code); }

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ LEnt ld_lent(const LEnt *p) {
    const uint4 x = __ldcg((const uint4 *)p);
    return LEnt{x.x, x.y, (int32_t)x.z, x.w};
}
__device__ __forceinline__ EHdr ld_ehdr(const EHdr *p) {
    const uint4 x = __ldcg((const uint4 *)p);
    return EHdr{x.x, x.y, (int32_t)x.z, x.w};
}
__device__ __forceinline__ void st_ehdr(EHdr *p, uint32_t slot_mask, uint32_t v, int kb, uint32_t lv) {
    __stcg((uint4 *)p, make_uint4(slot_mask, v, (uint32_t)kb, lv));
}

// 16 bases starting at base position p of a packed stream.
__device__ __forceinline__ uint32_t window16(const uint32_t *__restrict__ w, uint64_t p) {
    const uint64_t wi = p >> 4;
    const uint32_t sh = (uint32_t)(p & 15) * 2;
    const uint32_t lo = __ldg(w + wi), hi = __ldg(w + wi + 1);
    return __funnelshift_r(lo, hi, sh);
}

struct QCtx {
    const uint32_t *qw;   // this query's packed words (global, or staged in shared memory)
    int n;
    uint32_t ve;
    int ke;
    bool smem;            // qw points to shared memory (server kernel)
    bool free_end;        // the walk may end at any position of v_e (or anywhere: any_v)
    bool any_v;           // no end vertex
};

// End test of Alg. 1 on a diagonal just extended to offset j: the point (k + j, j)
// of v is the end point (|q|, |v_e|) of v_e; with a free walk end, any point of
// v_e on query position |q|; without an end vertex, any such point.
__device__ __forceinline__ bool at_end(const QCtx &q, uint32_t v, int k, int j, uint32_t lv) {
    if (k + j != q.n) return false;
    if (q.any_v) return true;
    return v == q.ve && (q.free_end || (uint32_t)j == lv);
}

// 16 query bases from position p: read-only cache for a batch staged before the
// launch, plain (shared-memory) loads for a query the CTA staged itself.
__device__ __forceinline__ uint32_t qwin(const QCtx &q, uint64_t p) {
    const uint64_t wi = p >> 4;
    const uint32_t sh = (uint32_t)(p & 15) * 2;
    uint32_t lo, hi;
    if (q.smem) {
        lo = q.qw[wi];
        hi = q.qw[wi + 1];
    } else {
        lo = __ldg(q.qw + wi);
        hi = __ldg(q.qw + wi + 1);
    }
    return __funnelshift_r(lo, hi, sh);
}

// LCP(q[i+1..|q|], v[j+1..|v|]) of Eq. 2 in 0-based positions: XOR of 16-base
// windows, the first differing base is the lowest set bit pair.
__device__ __forceinline__ int lcp(const QCtx &q, int i, const uint32_t *__restrict__ vw, int j,
                                   int lv) {
    const int maxl = min(q.n - i, lv - j);
    int l = 0;
    while (l < maxl) {
        const uint32_t x = qwin(q, (uint64_t)(i + l)) ^ window16(vw, (uint64_t)(j + l));
        if (x) {
            l += (__ffs(x) - 1) >> 1;
            break;
        }
        l += 16;
    }
    return min(l, maxl);
}

// The same LCP when the first window XOR `x` (bases i.. against j..) is already
// loaded, so that two diagonals can have their first windows in flight together.
__device__ __forceinline__ int lcp_finish(const QCtx &q, int i, const uint32_t *__restrict__ vw,
                                          int j, int maxl, uint32_t x) {
    int l = 0;
    while (l < maxl) {
        if (x) {
            l += (__ffs(x) - 1) >> 1;
            break;
        }
        l += 16;
        if (l >= maxl) break;
        x = qwin(q, (uint64_t)(i + l)) ^ window16(vw, (uint64_t)(j + l));
    }
    return min(l, maxl);
}

// Pruning mode: atomics on slab memory (always device global memory) issued in the
// global state space; the slab pointers come from shared memory, where the compiler
// no longer knows their space.
__device__ __forceinline__ uint32_t g_exch(uint32_t *p, uint32_t v) {
    uint32_t r;
    asm volatile("atom.global.exch.b32 %0, [%1], %2;" : "=r"(r) : "l"(p), "r"(v) : "memory");
    return r;
}
__device__ __forceinline__ long long g_max(long long *p, long long v) {
    long long r;
    asm volatile("atom.global.max.s64 %0, [%1], %2;" : "=l"(r) : "l"(p), "l"(v) : "memory");
    return r;
}
__device__ __forceinline__ unsigned long long g_cas(unsigned long long *p, unsigned long long c,
                                                    unsigned long long v) {
    unsigned long long r;
    asm volatile("atom.global.cas.b64 %0, [%1], %2, %3;" : "=l"(r) : "l"(p), "l"(c), "l"(v) : "memory");
    return r;
}
template <bool P, class T>
__device__ __forceinline__ T slab_max(T *p, T v) {
    if constexpr (P) return g_max(p, v);
    else return atomicMax(p, v);
}

__device__ __forceinline__ unsigned long long tile_key(uint32_t v, int kb) {
    return ((unsigned long long)v << 32) | (uint32_t)kb;
}

__device__ __forceinline__ uint32_t tile_hash(unsigned long long key, uint32_t mask) {
    return (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 32) & mask;
}

// find_or_insert's probe sequence when the key of its first slot h was already read
// (cur), so that the read can be issued ahead of other round trips.
template <bool P>
__device__ int find_or_insert_at(const Slab<P> &s, Sh &sh, unsigned long long key, uint32_t h,
                                 unsigned long long cur) {
    for (int probe = 0; probe < 256; ++probe) {
        if (probe > 0) cur = __ldcg(&s.slots[h].key);
        if (cur == key) return (int)h;
        if (cur == kEmptyKey) {
            unsigned long long prev;
            if constexpr (P) prev = g_cas(&s.slots[h].key, kEmptyKey, key);
            else prev = atomicCAS(&s.slots[h].key, kEmptyKey, key);
            if (prev == kEmptyKey) {
                const uint32_t t = atomicAdd(&sh.nt, 1u);
                s.touched[t] = h;   // t < cap: each claim takes a distinct empty slot
                if (t + 1 > (s.cap >> 1) + (s.cap >> 2)) set_err(sh, GWFA_ERR_CAPACITY);
                return (int)h;
            }
            if (prev == key) return (int)h;
        }
        h = (h + 1) & s.mask;
    }
    set_err(sh, GWFA_ERR_CAPACITY);
    return -1;
}

template <bool P>
__device__ int find_or_insert(const Slab<P> &s, Sh &sh, unsigned long long key) {
    const uint32_t h = tile_hash(key, s.mask);
    return find_or_insert_at(s, sh, key, h, __ldcg(&s.slots[h].key));
}

// Make lane `bit` of tile (slot, v, kb) live for the phase owning `regw`; the
// first lane to do so appends the tile to that phase's list.
__device__ __forceinline__ void reg_append(uint32_t *regw, LEnt *list, uint32_t *count,
                                           uint32_t cap, uint32_t slot, uint32_t v, int kb,
                                           uint32_t bit, Sh &sh) {
    if (atomicOr(regw, bit) == 0u) {
        const uint32_t i = atomicAdd(count, 1u);
        if (i < cap) __stcg((uint4 *)&list[i], make_uint4(slot, v, (uint32_t)kb, 0u));
        else set_err(sh, GWFA_ERR_CAPACITY);
    }
}

// Dynamic work distribution inside a phase: lane 0 of a warp claims the next
// 4 x `step` entries for the warp's four groups (group g of the warp takes entries
// [base + g step, base + (g + 1) step)), so a warp held up by a long exact-match run
// or spill chain does not stall the others at the phase barrier, and the four groups
// run the same iterations in step.  Every lane of the warp calls it.
__device__ __forceinline__ uint32_t warp_claim(uint32_t *ctr, uint32_t step) {
    uint32_t e = 0;
    if ((threadIdx.x & 31) == 0) e = atomicAdd(ctr, 4u * step);
    return __shfl_sync(0xFFFFFFFFu, e, 0);
}



// Exact mode: diagonal (v, k) reached |v| (Alg. 2 arc loop).  Offset 0 goes to
// (u, k + |v|) for every arc (v, u) where it is absent; a diagonal this thread
// inserts is extended by this thread at once, depth first, with its own arcs in
// turn.  Only when the small stack is full does a won diagonal go to the spill
// list of the next round instead.
__device__ void spill_dfs(const DevGraph &g, const Slab<false> &s, Sh &sh, const QCtx &q,
                          uint32_t arc0, uint32_t arc1, int ku0, int next_par, LEnt *next_list,
                          uint32_t *next_count) {
    uint32_t st_slot[kStack], st_u[kStack];
    int st_k[kStack];
    int top = 0;
    uint32_t a0 = arc0, a1 = arc1;
    int ku = ku0;
    for (;;) {
        for (uint32_t a = a0; a < a1; ++a) {
            const uint32_t u = __ldg(&g.arc_dst[a]);
            const int su = find_or_insert(s, sh, tile_key(u, ku >> 3));
            if (su < 0) return;
            const int prev = atomicMax(&s.slots[su].vals[ku & 7], 0);
            if (prev < 0) {
                atomicAdd(&sh.spills32, 1u);
                if (top < kStack) {
                    st_slot[top] = (uint32_t)su;
                    st_u[top] = u;
                    st_k[top] = ku;
                    ++top;
                } else {
                    reg_append(&s.slots[su].reg[next_par], next_list, next_count, s.cap, (uint32_t)su, u, ku >> 3,
                               1u << (ku & 7), sh);
                }
            }
        }
        if (top == 0) return;
        --top;
        const uint32_t su = st_slot[top], u = st_u[top];
        const int k = st_k[top];
        const uint4 vi = __ldg(&g.vinfo[u]);
        const int l = lcp(q, k, g.words + vi.x, 0, (int)vi.y);
        __stcg(&s.slots[su].vals[k & 7], l);
        const uint32_t eidx = atomicAdd(&sh.ne, 1u);
        atomicAdd(&sh.score_cells, 1u);
        if (eidx < s.cap) {
            st_ehdr(&s.elist[eidx].hdr, su | ((1u << (k & 7)) << 24), u, k >> 3, vi.y);
            __stcg(&s.elist[eidx].vals[k & 7], l);
        } else {
            set_err(sh, GWFA_ERR_CAPACITY);
        }
        if (at_end(q, u, k, l, vi.y)) sh.found = 1;
        if ((uint32_t)l == vi.y) {
            a0 = vi.z;
            a1 = vi.w;
            ku = k + (int)vi.y;
        } else {
            a0 = a1 = 0;
        }
    }
}

// One extension round over `list` in exact mode.  Each 8-lane group takes
// U tiles per iteration and keeps their dependency chains (list entry ->
// mask, offsets, vertex info -> first LCP window) in flight together.
template <int U>
__device__ void extend_round_exact(const DevGraph &g, const Slab<false> &s, Sh &sh, const QCtx &q,
                                   const LEnt *list, uint32_t n_list, int par, int next_par,
                                   LEnt *next_list, uint32_t *next_count, uint32_t *claim) {
    const int ln = threadIdx.x & 7;
    const unsigned gmask = 0xFFu << (threadIdx.x & 24);
    for (;;) {
        const uint32_t wb = warp_claim(claim, (uint32_t)U);
        if (wb >= n_list) break;
        const uint32_t e0 = wb + ((threadIdx.x & 31) >> 3) * (uint32_t)U;
        if (e0 >= n_list) continue;   // nothing left for this group in the warp's claim
        const uint32_t cnt = min((uint32_t)U, n_list - e0);   // uniform within the group
        LEnt ent[U];
        uint32_t m[U];
        int val[U];
        uint2 vi[U];   // label word, |v| (the arc range is reloaded for the rare spill)
#pragma unroll
        for (int u = 0; u < U; ++u) {
            ent[u] = (u == 0 || (uint32_t)u < cnt) ? ld_lent(&list[e0 + u]) : ent[0];
            m[u] = 0u;
            if (ln == 0 && (uint32_t)u < cnt) m[u] = atomicExch(&s.slots[ent[u].slot].reg[par], 0u);
            val[u] = __ldcg(&s.slots[ent[u].slot].vals[ln]);
            vi[u] = __ldg((const uint2 *)&g.vinfo[ent[u].v]);
        }
        uint32_t eidx = 0, pop = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            m[u] = __shfl_sync(gmask, m[u], 0, 8);
            pop += __popc(m[u]);
        }
        if (ln == 0) {
            eidx = atomicAdd(&sh.ne, cnt);
            atomicAdd(&sh.score_cells, pop);
        }
        eidx = __shfl_sync(gmask, eidx, 0, 8);
        bool live[U];
        int k[U], maxl[U];
        uint32_t x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            live[u] = (m[u] >> ln) & 1u;
            k[u] = ent[u].kb * kTile + ln;
            maxl[u] = 0;
            x[u] = 0;
            if (live[u]) {
                const int i = k[u] + val[u];
                maxl[u] = min(q.n - i, (int)vi[u].y - val[u]);
                if (maxl[u] > 0)
                    x[u] = qwin(q, (uint64_t)i) ^ window16(g.words + vi[u].x, (uint64_t)val[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if ((uint32_t)u >= cnt) break;
            if (live[u]) {
                val[u] += lcp_finish(q, k[u] + val[u], g.words + vi[u].x, val[u], maxl[u], x[u]);
                __stcg(&s.slots[ent[u].slot].vals[ln], val[u]);
                if (at_end(q, ent[u].v, k[u], val[u], vi[u].y)) sh.found = 1;
            }
            const uint32_t ei = eidx + u;
            if (ei < s.cap) {
                if (ln == 0) st_ehdr(&s.elist[ei].hdr, ent[u].slot | (m[u] << 24), ent[u].v, ent[u].kb, vi[u].y);
                __stcg(&s.elist[ei].vals[ln], live[u] ? val[u] : -1);
            } else if (ln == 0) {
                set_err(sh, GWFA_ERR_CAPACITY);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if ((uint32_t)u >= cnt) break;
            if (live[u] && (uint32_t)val[u] == vi[u].y) {
                const uint4 full = __ldg(&g.vinfo[ent[u].v]);
                spill_dfs(g, s, sh, q, full.z, full.w, k[u] + (int)vi[u].y, next_par, next_list, next_count);
            }
        }
    }
}

// GwfPushTrace (Alg. 5): record "vertex v, reached with trace t" and return its
// index in T.  Unlike Alg. 5, equal (v, t) pairs are not merged through a map:
// T then holds one entry per spilling diagonal, which bounds it by the spill count
// and gives the same walk.
__device__ __forceinline__ uint32_t push_trace(const Slab<true> &s, Sh &sh, uint32_t v, uint32_t t) {
    const uint32_t idx = atomicAdd(&sh.tlen, 1u);
    if (idx >= 2 * s.cap || idx >= kNoTrace) {
        set_err(sh, GWFA_ERR_CAPACITY);
        return kNoTrace;
    }
    __stcg(&s.trace[idx], make_uint2(v, t));
    return idx;
}

// One extension round over `list` in pruning mode.  Spills are recorded, not
// applied: apply_spill_requests runs after the round's barrier, so a spill can
// never touch a diagonal that was present before the round (Alg. 2's presence
// test) and same-round spills into one diagonal merge by the larger walk base.
__device__ void extend_round_prune(const DevGraph &g, const Slab<true> &s, Sh &sh, const QCtx &q,
                                   const LEnt *list, uint32_t n_list, int par, uint32_t *req_count,
                                   uint32_t *claim, bool traceback) {
    const int ln = threadIdx.x & 7;
    const unsigned gmask = 0xFFu << (threadIdx.x & 24);
    for (;;) {
        const uint32_t wb = warp_claim(claim, 1u);
        if (wb >= n_list) break;
        const uint32_t e = wb + ((threadIdx.x & 31) >> 3);
        if (e >= n_list) continue;
        const LEnt ent = ld_lent(&list[e]);
        uint32_t m = 0, eidx = 0;
        if (ln == 0) m = g_exch(&s.slots[ent.slot].reg[par], 0u);
        long long val = __ldcg(&s.slots[ent.slot].vals[ln]);
        const uint2 vi = __ldg((const uint2 *)&g.vinfo[ent.v]);   // label word, |v|
        const uint32_t tr = traceback ? __ldcg(&s.slots[ent.slot].trace[ln]) : 0u;
        m = __shfl_sync(gmask, m, 0, 8);
        if (ln == 0) {
            eidx = atomicAdd(&sh.ne, 1u);
            atomicAdd(&sh.score_cells, (uint32_t)__popc(m));
        }
        eidx = __shfl_sync(gmask, eidx, 0, 8);
        const int k = ent.kb * kTile + ln;
        const bool live = (m >> ln) & 1u;
        unsigned long long a = 0;
        if (live) {
            const int j = pj(val);
            const int i = k + j;
            const int j2 = j + lcp(q, i, g.words + vi.x, j, (int)vi.y);
            val = pk(j2, kTagSettled, pbase(val));
            __stcg(&s.slots[ent.slot].vals[ln], val);
            if (at_end(q, ent.v, k, j2, vi.y)) {
                sh.found = 1;
                // one 64-bit store, so that the vertex and its trace stay a pair when
                // several diagonals reach a free end in the same score
                sh.end_vp = ((unsigned long long)ent.v << 32) | tr;
            }
            a = (unsigned long long)(k + j2) + pbase(val) + (unsigned)j2;   // a = i + W~ (Alg. 4)
            if ((uint32_t)j2 == vi.y) {
                // the spilled diagonals get the walk base past v and, with traceback,
                // the index of the T entry "left v with this trace" (Alg. 5)
                const uint32_t nb = pbase(val) + vi.y;
                if (nb > kBaseMask) set_err(sh, GWFA_ERR_CAPACITY);
                const uint32_t t = traceback ? push_trace(s, sh, ent.v, tr) : 0u;
                const uint32_t r = atomicAdd(req_count, 1u);
                if (r < s.cap) {
                    const uint4 full = __ldg(&g.vinfo[ent.v]);   // the arc range, for the rare spill
                    __stcg(&s.req[r], make_int4(k + (int)vi.y, (int)nb, (int)full.z, (int)full.w));
                    if (traceback) __stcg(&s.reqt[r], t);
                } else {
                    set_err(sh, GWFA_ERR_CAPACITY);
                }
            }
        }
        for (int o = 4; o >= 1; o >>= 1) {
            const unsigned long long b = __shfl_xor_sync(gmask, a, o, 8);
            a = b > a ? b : a;
        }
        if (ln == 0 && a > 0) atomicMax(&sh.amax, a);
        if (eidx < s.cap) {
            if (ln == 0) st_ehdr(&s.elist[eidx].hdr, ent.slot | (m << 24), ent.v, ent.kb, vi.y);
            __stcg(&s.elist[eidx].vals[ln], live ? val : -1ll);
            if (traceback) __stcg(&s.elist[eidx].trace[ln], tr);
        } else if (ln == 0) {
            set_err(sh, GWFA_ERR_CAPACITY);
        }
    }
}

// Pruning mode, second half of a round: offset 0 with walk base nb on (u, ku)
// for every recorded spill; the inserted diagonals form the next round's list.
__device__ void apply_spill_requests(const DevGraph &g, const Slab<true> &s, Sh &sh, uint32_t n_req,
                                     int next_par, LEnt *next_list, uint32_t *next_count) {
    const uint32_t nr = min(n_req, s.cap);
    for (uint32_t r = threadIdx.x; r < nr; r += blockDim.x) {
        const int4 rq = __ldcg(&s.req[r]);
        const int ku = rq.x;
        const long long cand = pk(0, kTagPend, (uint32_t)rq.y);
        for (uint32_t a = (uint32_t)rq.z; a < (uint32_t)rq.w; ++a) {
            const uint32_t u = __ldg(&g.arc_dst[a]);
            const int su = find_or_insert(s, sh, tile_key(u, ku >> 3));
            if (su < 0) return;
            const long long prev = g_max(&s.slots[su].vals[ku & 7], cand);
            if (prev < 0) {
                atomicAdd(&sh.visited32, 1u);
                atomicAdd(&sh.spills32, 1u);
                __stcg(&s.slots[su].trace[ku & 7], 0u);   // set by resolve_spill_traces
                reg_append(&s.slots[su].reg[next_par], next_list, next_count, s.cap, (uint32_t)su, u, ku >> 3,
                           1u << (ku & 7), sh);
            }
        }
    }
}

// Traceback with pruning: after apply_spill_requests (and a barrier) every diagonal
// a spill inserted in this round holds the largest base among its spills, still
// tagged pending; each request whose base is that one offers its T index and the
// largest index wins (any of them is a walk of that base, so the choice only has to
// be deterministic).
__device__ void resolve_spill_traces(const DevGraph &g, const Slab<true> &s, Sh &sh, uint32_t n_req) {
    const uint32_t nr = min(n_req, s.cap);
    for (uint32_t r = threadIdx.x; r < nr; r += blockDim.x) {
        const int4 rq = __ldcg(&s.req[r]);
        const int ku = rq.x;
        const long long cand = pk(0, kTagPend, (uint32_t)rq.y);
        const uint32_t t = __ldcg(&s.reqt[r]);
        for (uint32_t a = (uint32_t)rq.z; a < (uint32_t)rq.w; ++a) {
            const int su = find_or_insert(s, sh, tile_key(__ldg(&g.arc_dst[a]), ku >> 3));
            if (su < 0) return;
            if (__ldcg(&s.slots[su].vals[ku & 7]) == cand) atomicMax(&s.slots[su].trace[ku & 7], t);
        }
    }
}

// Pruning mode: the merge of `cand` replaced `prev` and was the first of this
// GwfExpand to do so (every offset is settled when GwfExpand starts, so the first
// fresh value is the first change).
__device__ __forceinline__ bool first_fresh(long long prev, long long cand) {
    return cand > prev && ((prev >> 30) & 3) != kTagFresh;
}

// Offer value `cand` to lane `ln` of tile (slot, v, kb): GwfExpand's max-merge
// into H~; the lane joins the next Q if its offset strictly improved.
template <bool P>
__device__ __forceinline__ void offer_done(const Slab<P> &s, Sh &sh, uint32_t slot, uint32_t v, int kb,
                                           int ln, typename VT<P>::T cand, typename VT<P>::T prev, int par,
                                           uint32_t *qcount, bool traceback) {
    if constexpr (P) {
        if (prev < 0) atomicAdd(&sh.visited32, 1u);
        if (traceback && first_fresh(prev, cand)) __stcg(&s.slots[slot].trace[ln], 0u);
    }
    if (pj(prev) < pj(cand)) reg_append(&s.slots[slot].reg[par], s.qlist, qcount, s.cap, slot, v, kb, 1u << ln, sh);
}

template <bool P>
__device__ __forceinline__ void offer(const Slab<P> &s, Sh &sh, uint32_t slot, uint32_t v, int kb,
                                      int ln, typename VT<P>::T cand, int par, uint32_t *qcount, bool traceback) {
    const typename VT<P>::T prev = slab_max<P>(&s.slots[slot].vals[ln], cand);
    offer_done<P>(s, sh, slot, v, kb, ln, cand, prev, par, qcount, traceback);
}

// GwfExpand (Alg. 3) over the extended frontier, with GwfPrune (Alg. 4) applied
// to the sources on the way in.  U snapshot entries per group and
// iteration: their candidate max-merges are issued together before any registration.
template <bool P, int U>
__device__ void expand_all(const Slab<P> &s, Sh &sh, const QCtx &q, uint32_t n_e, bool prune_on,
                           long long amax, int max_lag, int par, uint32_t *qcount, uint32_t *claim,
                           bool traceback) {
    using T = typename VT<P>::T;
    const int ln = threadIdx.x & 7;
    const unsigned gmask = 0xFFu << (threadIdx.x & 24);
    const uint32_t ne = min(n_e, s.cap);
    for (;;) {
        const uint32_t wb = warp_claim(claim, (uint32_t)U);
        if (wb >= ne) break;
        const uint32_t base = wb + ((threadIdx.x & 31) >> 3) * (uint32_t)U;
        if (base >= ne) continue;
        bool valid[U], ins[U], del[U];
        EHdr h[U];
        T c_ins[U], c_del[U], cand[U], prev[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t e = base + u;
            valid[u] = e < ne;
            h[u] = EHdr{0u, 0u, 0, 0u};
            T val = (T)-1;
            if (valid[u]) {
                h[u] = ld_ehdr(&s.elist[e].hdr);
                val = __ldcg(&s.elist[e].vals[ln]);
            }
            const uint32_t m = h[u].slot_mask >> 24;
            bool act = valid[u] && ((m >> ln) & 1u);
            const int k = h[u].kb * kTile + ln;
            const int j = act ? pj(val) : 0;
            const int i = k + j;
            const uint32_t b = pbase(val);
            if (P && act && prune_on) {
                const long long a = (long long)i + (long long)b + j;
                if (amax - a >= (long long)max_lag) {
                    act = false;
                    atomicAdd(&sh.pruned32, 1u);
                }
            }
            ins[u] = act && i < q.n;                 // (k+1, j)
            del[u] = act && j < (int)h[u].lv;        // (k-1, j+1)
            const bool mis = ins[u] && j < (int)h[u].lv;   // (k, j+1)
            T c_mis;
            if constexpr (P) {
                c_ins[u] = ins[u] ? pk(j, kTagFresh, b) : -1ll;
                c_del[u] = del[u] ? pk(j + 1, kTagFresh, b) : -1ll;
                c_mis = mis ? pk(j + 1, kTagFresh, b) : -1ll;
            } else {
                c_ins[u] = ins[u] ? j : -1;
                c_del[u] = del[u] ? j + 1 : -1;
                c_mis = mis ? j + 1 : -1;
            }
            T from_left = __shfl_up_sync(gmask, c_ins[u], 1, 8);
            T from_right = __shfl_down_sync(gmask, c_del[u], 1, 8);
            if (ln == 0) from_left = (T)-1;
            if (ln == 7) from_right = (T)-1;
            cand[u] = c_mis;
            if (from_left > cand[u]) cand[u] = from_left;
            if (from_right > cand[u]) cand[u] = from_right;
        }
        // the neighbour tile a boundary lane leaves for (insertion from lane 7, deletion
        // from lane 0): its first hash read goes out before this tile's merges
        unsigned long long nkey[U], ncur[U];
        uint32_t nh[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool out = valid[u] && ((ln == 7 && ins[u]) || (ln == 0 && del[u]));
            nkey[u] = tile_key(h[u].v, h[u].kb + (ln == 7 ? 1 : -1));
            nh[u] = tile_hash(nkey[u], s.mask);
            ncur[u] = out ? __ldcg(&s.slots[nh[u]].key) : 0ull;
        }
        // a boundary lane whose early read found the neighbour tile merges into it
        // together with this tile's merges
        bool near[U];
        T nprev[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            prev[u] = (T)0x7FFFFFFF;
            if (valid[u] && cand[u] >= 0)
                prev[u] = slab_max<P>(&s.slots[h[u].slot_mask & 0xFFFFFFu].vals[ln], cand[u]);
            near[u] = ncur[u] == nkey[u] && valid[u] && ((ln == 7 && ins[u]) || (ln == 0 && del[u]));
            nprev[u] = 0;
            if (near[u]) nprev[u] = slab_max<P>(&s.slots[nh[u]].vals[7 - ln], ln == 7 ? c_ins[u] : c_del[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!(valid[u] && cand[u] >= 0)) continue;
            if constexpr (P) {
                if (prev[u] < 0) atomicAdd(&sh.visited32, 1u);   // exact mode counts at query end
            }
            if constexpr (P) {
                if (traceback && first_fresh(prev[u], cand[u]))
                    __stcg(&s.slots[h[u].slot_mask & 0xFFFFFFu].trace[ln], 0u);
            }
            if (pj(prev[u]) < pj(cand[u]))
                reg_append(&s.slots[h[u].slot_mask & 0xFFFFFFu].reg[par], s.qlist, qcount, s.cap,
                           h[u].slot_mask & 0xFFFFFFu, h[u].v,
                           h[u].kb, 1u << ln, sh);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (valid[u] && ln == 7 && ins[u]) {   // insertion leaves the tile: (v, 8(kb+1))
                if (near[u]) {
                    offer_done<P>(s, sh, nh[u], h[u].v, h[u].kb + 1, 0, c_ins[u], nprev[u], par, qcount, traceback);
                } else {
                    const int t = find_or_insert_at(s, sh, nkey[u], nh[u], ncur[u]);
                    if (t >= 0) offer<P>(s, sh, (uint32_t)t, h[u].v, h[u].kb + 1, 0, c_ins[u], par, qcount, traceback);
                }
            }
            if (valid[u] && ln == 0 && del[u]) {   // deletion leaves the tile: (v, 8 kb - 1)
                if (near[u]) {
                    offer_done<P>(s, sh, nh[u], h[u].v, h[u].kb - 1, 7, c_del[u], nprev[u], par, qcount, traceback);
                } else {
                    const int t = find_or_insert_at(s, sh, nkey[u], nh[u], ncur[u]);
                    if (t >= 0) offer<P>(s, sh, (uint32_t)t, h[u].v, h[u].kb - 1, 7, c_del[u], par, qcount, traceback);
                }
            }
        }
    }
}

// Traceback with pruning, after GwfExpand's merge (and a barrier): every diagonal
// the merge raised holds the largest candidate (offset, base), tagged fresh; each
// candidate equal to it offers the trace index of its source, and the largest
// index wins (sources of equal offset and base are equally good predecessors).
// The candidates and the pruning of their sources are recomputed as in expand_all.
__device__ void resolve_expand_traces(const Slab<true> &s, Sh &sh, const QCtx &q, uint32_t n_e, bool prune_on,
                                      long long amax, int max_lag, uint32_t *claim) {
    const int ln = threadIdx.x & 7;
    const unsigned gmask = 0xFFu << (threadIdx.x & 24);
    const uint32_t ne = min(n_e, s.cap);
    for (;;) {
        const uint32_t wb = warp_claim(claim, 1u);
        if (wb >= ne) break;
        const uint32_t e = wb + ((threadIdx.x & 31) >> 3);
        if (e >= ne) continue;
        const EHdr h = ld_ehdr(&s.elist[e].hdr);
        const long long val = __ldcg(&s.elist[e].vals[ln]);
        const uint32_t tr = __ldcg(&s.elist[e].trace[ln]);
        const uint32_t slot = h.slot_mask & 0xFFFFFFu;
        bool act = (h.slot_mask >> (24 + ln)) & 1u;
        const int k = h.kb * kTile + ln;
        const int j = act ? pj(val) : 0;
        const int i = k + j;
        const uint32_t b = pbase(val);
        if (act && prune_on && amax - ((long long)i + (long long)b + j) >= (long long)max_lag) act = false;
        const bool ins = act && i < q.n;
        const bool del = act && j < (int)h.lv;
        const bool mis = ins && j < (int)h.lv;
        const long long c_ins = ins ? pk(j, kTagFresh, b) : -1ll;
        const long long c_del = del ? pk(j + 1, kTagFresh, b) : -1ll;
        long long from_left = __shfl_up_sync(gmask, c_ins, 1, 8);
        long long from_right = __shfl_down_sync(gmask, c_del, 1, 8);
        const uint32_t t_left = __shfl_up_sync(gmask, tr, 1, 8);
        const uint32_t t_right = __shfl_down_sync(gmask, tr, 1, 8);
        if (ln == 0) from_left = -1;
        if (ln == 7) from_right = -1;
        if (mis || from_left >= 0 || from_right >= 0) {
            const long long cur = __ldcg(&s.slots[slot].vals[ln]);
            if (mis && cur == pk(j + 1, kTagFresh, b)) atomicMax(&s.slots[slot].trace[ln], tr);
            if (from_left >= 0 && cur == from_left) atomicMax(&s.slots[slot].trace[ln], t_left);
            if (from_right >= 0 && cur == from_right) atomicMax(&s.slots[slot].trace[ln], t_right);
        }
        if (ln == 7 && ins) {   // insertion left the tile: (v, 8(kb+1)), lane 0
            const int t = find_or_insert(s, sh, tile_key(h.v, h.kb + 1));
            if (t >= 0 && __ldcg(&s.slots[t].vals[0]) == c_ins) atomicMax(&s.slots[t].trace[0], tr);
        }
        if (ln == 0 && del) {   // deletion left the tile: (v, 8 kb - 1), lane 7
            const int t = find_or_insert(s, sh, tile_key(h.v, h.kb - 1));
            if (t >= 0 && __ldcg(&s.slots[t].vals[7]) == c_del) atomicMax(&s.slots[t].trace[7], tr);
        }
    }
}

template <bool P>
__device__ void wipe_touched(const Slab<P> &s, uint32_t nt) {
    using T = typename VT<P>::T;
    nt = min(nt, s.cap);
    for (uint32_t t = threadIdx.x; t < nt * kTile; t += blockDim.x) {
        const uint32_t slot = __ldcg(&s.touched[t / kTile]);
        __stcg(&s.slots[slot].vals[t % kTile], (T)-1);
        if (t % kTile == 0) {
            __stcg(&s.slots[slot].key, kEmptyKey);
            __stcg((unsigned long long *)s.slots[slot].reg, 0ull);
        }
    }
}

// Memory bound on H~ (pruning mode, called every evict_every scores right after
// GwfExpand): the lanes in the new Q (registered in parity `par`) and those whose
// anti-diagonal a = i + W~ lags this score's a_max by less than `lag` are kept, the
// others are removed (sh.evicted).  The tiles with a kept lane are staged in the
// frontier-snapshot list, which is free between scores; the table is wiped through
// the touched list and they are inserted again, and Q is rebuilt with their new
// slots.  A removed diagonal may be inserted again later, like any absent one.
__device__ void evict_behind(const Slab<true> &s, Sh &sh, long long amax, int lag, int par,
                             uint32_t *qcount) {
    const uint32_t nt = min(sh.nt, s.cap);
    if (threadIdx.x == 0) sh.nsurv = 0;
    __syncthreads();
    unsigned long long ev = 0;
    for (uint32_t t = threadIdx.x; t < nt; t += blockDim.x) {
        const uint32_t slot = __ldcg(&s.touched[t]);
        const unsigned long long key = __ldcg(&s.slots[slot].key);
        const uint32_t regw = __ldcg(&s.slots[slot].reg[par]);
        const int kb = (int)(uint32_t)(key & 0xFFFFFFFFull);
        long long v8[kTile];
        uint32_t keep = 0;
#pragma unroll
        for (int ln = 0; ln < kTile; ++ln) {
            v8[ln] = __ldcg(&s.slots[slot].vals[ln]);
            if (v8[ln] < 0) continue;
            const int j = pj(v8[ln]);
            const long long a = (long long)(kb * kTile + ln) + 2ll * j + (long long)pbase(v8[ln]);
            if (((regw >> ln) & 1u) || amax - a < (long long)lag) keep |= 1u << ln;
            else ++ev;
        }
        if (keep) {
            const uint32_t i = atomicAdd(&sh.nsurv, 1u);   // i < nt <= cap
            st_ehdr(&s.elist[i].hdr, regw, (uint32_t)(key >> 32), kb, 0u);
#pragma unroll
            for (int ln = 0; ln < kTile; ++ln)
                __stcg(&s.elist[i].vals[ln], ((keep >> ln) & 1u) ? v8[ln] : -1ll);
        }
    }
    if (ev) atomicAdd(&sh.evicted, ev);
    __syncthreads();
    wipe_touched<true>(s, nt);
    if (threadIdx.x == 0) {
        sh.nt = 0;
        *qcount = 0;
    }
    __syncthreads();
    const uint32_t ns = sh.nsurv;
    for (uint32_t i = threadIdx.x; i < ns; i += blockDim.x) {
        const EHdr h = ld_ehdr(&s.elist[i].hdr);
        const int slot = find_or_insert(s, sh, tile_key(h.v, h.kb));
        if (slot < 0) continue;
#pragma unroll
        for (int ln = 0; ln < kTile; ++ln) __stcg(&s.slots[slot].vals[ln], __ldcg(&s.elist[i].vals[ln]));
        if (h.slot_mask) {   // part of the new Q
            __stcg(&s.slots[slot].reg[par], h.slot_mask);
            const uint32_t qi = atomicAdd(qcount, 1u);
            if (qi < s.cap) __stcg((uint4 *)&s.qlist[qi], make_uint4((uint32_t)slot, h.v, (uint32_t)h.kb, 0u));
            else set_err(sh, GWFA_ERR_CAPACITY);
        }
    }
    __syncthreads();
}

template <bool P>
__device__ void align_one(const TierArgs &A, const Slab<P> &s, Sh &sh, uint32_t qid) {
    const DevGraph &g = A.g;
    const uint64_t qo = A.q_off[qid];
    const int n = (int)(A.q_off[qid + 1] - qo);
    QCtx q;
    q.qw = A.qwords + (qo >> 4) + qid;
    q.n = n;
    q.smem = A.q_smem != 0;
    const uint32_t vs = A.v_s[qid];
    q.ve = A.v_e[qid];
    int pre = 0;
    if (A.qstatus) pre = A.qstatus[qid];
    q.any_v = (A.ends & GWFA_EXTEND) != 0;
    q.free_end = (A.ends & (GWFA_FREE_END | GWFA_EXTEND)) != 0;
    if (q.any_v) q.ve = vs;   // no end vertex: v_e is not read
    if (!pre && (vs >= g.nv || q.ve >= g.nv)) pre = GWFA_ERR_INVALID;
    if (pre) {
        if (threadIdx.x == 0) {
            gwfa_result r = {};
            r.status = pre;
            r.edit_distance = -1;
            A.out[qid] = r;
        }
        return;
    }
    q.ke = n - (int)__ldg(&g.vinfo[q.ve]).y;
    // Alg. 1 initialisation: H~_{v_s,0} <- 0, Q <- [(v_s, 0)], d <- 0
    if (threadIdx.x == 0) {
        sh.t_start = globaltimer_ns();
        for (int i = 0; i < 6; ++i) sh.st[i] = 0;
        sh.err = 0;
        sh.nt = 0;
        sh.cells = sh.visited = sh.pruned = sh.spills = sh.evicted = 0;
        sh.spills32 = sh.visited32 = sh.pruned32 = 0;
        sh.peak = 0;
        sh.nq[0] = sh.nq[1] = 0;
        sh.claim[0] = sh.claim[1] = sh.claim[2] = 0;
        sh.tlen = 0;
        sh.end_vp = ((unsigned long long)q.ve << 32) | kNoTrace;
        const int slot = find_or_insert(s, sh, tile_key(vs, 0));
        if (slot >= 0) {
            typename VT<P>::T v0;
            if constexpr (P) {
                v0 = pk(0, kTagFresh, 0u);
                s.slots[slot].trace[0] = kNoTrace;
            } else {
                v0 = 0;
            }
            s.slots[slot].vals[0] = v0;
            if constexpr (P) sh.visited = 1;
            reg_append(&s.slots[slot].reg[1], s.qlist, &sh.nq[0], s.cap, (uint32_t)slot, vs, 0, 1u, sh);
        }
    }
    __syncthreads();
    if (A.ends & GWFA_FREE_START) {
        // free walk start (Sec. 2.1 variant): query position 0 also faces every
        // position j of v_s, i.e. the diagonals (v_s, -j) start with offset j
        const int lvs = (int)__ldg(&g.vinfo[vs]).y;
        const int ntile = (lvs + kTile - 1) / kTile;   // tiles kb = -1 .. -ntile
        for (int t = threadIdx.x; t < ntile; t += blockDim.x) {
            const int kb = -1 - t;
            uint32_t bits = 0;
            for (int ln = 0; ln < kTile; ++ln)
                if (kb * kTile + ln >= -lvs) bits |= 1u << ln;
            const int slot = find_or_insert(s, sh, tile_key(vs, kb));
            if (slot < 0) continue;
            for (int ln = 0; ln < kTile; ++ln) {
                if (!((bits >> ln) & 1u)) continue;
                const int j = -(kb * kTile + ln);
                if constexpr (P) {
                    s.slots[slot].vals[ln] = pk(j, kTagFresh, 0u);
                    s.slots[slot].trace[ln] = kNoTrace;
                } else {
                    s.slots[slot].vals[ln] = j;
                }
            }
            if constexpr (P) atomicAdd(&sh.visited, (unsigned long long)__popc(bits));
            reg_append(&s.slots[slot].reg[1], s.qlist, &sh.nq[0], s.cap, (uint32_t)slot, vs, kb, bits, sh);
        }
        __syncthreads();
    }

    uint32_t phase = 1;   // parity (phase & 1) of the reg words of the tiles in Q
    uint32_t cstep = 0;   // processing phases so far: phase number c claims with claim[c % 3]
    int d = 0;
    int status = 0;
    int failed = 0;
    for (;;) {
        // ---- GwfExtend (Alg. 2)
        if (threadIdx.x == 0) {
            sh.ne = 0;
            sh.score_cells = 0;
            sh.found = 0;
            sh.amax = 0;
            sh.ns[1] = 0;
            sh.nreq[0] = 0;
            sh.nq[(d + 1) & 1] = 0;
        }
        __syncthreads();
        const LEnt *list = s.qlist;
        uint32_t n_list = min(sh.nq[d & 1], s.cap);
        if (A.stats && threadIdx.x == 0) sh.t_phase = globaltimer_ns();
        for (int round = 0;; ++round) {
            if (A.stats && threadIdx.x == 0) {
                sh.st[2]++;
                sh.st[3] += n_list;
            }
            const uint32_t next_phase = phase + 1;
            LEnt *next_list = s.slist[(round + 1) & 1];
            // round r fills ns[(r+1)%3] and clears ns[(r+2)%3] for round r+1; the
            // cleared counter was last read before the previous round's barrier
            uint32_t *next_count = &sh.ns[(round + 1) % 3];
            // processing phase c claims with claim[c % 3] and clears the two others for
            // the next phase; both were last used before this phase's barrier
            if (threadIdx.x == 0) {
                sh.ns[(round + 2) % 3] = 0;
                sh.claim[(cstep + 1) % 3] = 0;
                sh.claim[(cstep + 2) % 3] = 0;
            }
            uint32_t *claim = &sh.claim[cstep % 3];
            ++cstep;
            if constexpr (P) {
                extend_round_prune(g, s, sh, q, list, n_list, phase & 1, &sh.nreq[round & 1], claim,
                                   A.traceback != 0);
                __syncthreads();
                if (threadIdx.x == 0) sh.nreq[(round + 1) & 1] = 0;
                apply_spill_requests(g, s, sh, sh.nreq[round & 1], next_phase & 1, next_list,
                                     next_count);
                if (A.traceback) {
                    __syncthreads();
                    resolve_spill_traces(g, s, sh, sh.nreq[round & 1]);
                }
            } else {
                extend_round_exact<kGroupTiles>(g, s, sh, q, list, n_list, phase & 1, next_phase & 1,
                                                next_list, next_count, claim);
            }
            // every exit decision comes from a barrier reduction: sh.err may be set by
            // threads that already run the next phase, so it is never re-read for control
            failed = __syncthreads_or(sh.err != 0);
            const uint32_t ns = *next_count;
            phase = next_phase;
            if (failed || ns == 0) break;
            list = next_list;
            n_list = min(ns, s.cap);
        }
        if (threadIdx.x == 0) {
            sh.cells += sh.score_cells;
            sh.spills += atomicExch(&sh.spills32, 0u);
            sh.visited += atomicExch(&sh.visited32, 0u);
            sh.pruned += atomicExch(&sh.pruned32, 0u);
            sh.peak = max(sh.peak, sh.score_cells);
        }
        if (A.stats && threadIdx.x == 0) {
            const unsigned long long t = globaltimer_ns();
            sh.st[0] += t - sh.t_phase;
            sh.t_phase = t;
            sh.st[4] += sh.ne;
            sh.st[5] = max(sh.st[5], (unsigned long long)sh.ne);
        }
        if (failed) break;
        // end test of Alg. 1
        if (sh.found) break;
        if (A.max_score >= 0 && d >= A.max_score) { status = GWFA_ERR_SCORE_LIMIT; break; }
        d = d + 1;
        // ---- GwfPrune (Alg. 4) folded into the sources of GwfExpand (Alg. 3)
        const long long amax = (long long)sh.amax;
        const bool prune_on = P && A.max_lag > 0 && amax > (long long)A.max_lag;
        phase = phase + 1;
        if (threadIdx.x == 0) {
            sh.claim[(cstep + 1) % 3] = 0;
            sh.claim[(cstep + 2) % 3] = 0;
        }
        uint32_t *claim = &sh.claim[cstep % 3];
        ++cstep;
        expand_all<P, kGroupTiles>(s, sh, q, sh.ne, prune_on, amax, A.max_lag, phase & 1, &sh.nq[d & 1],
                                   claim, A.traceback != 0);
        failed = __syncthreads_or(sh.err != 0);
        if constexpr (P) {
            if (A.traceback && !failed) {
                if (threadIdx.x == 0) {
                    sh.claim[(cstep + 1) % 3] = 0;
                    sh.claim[(cstep + 2) % 3] = 0;
                }
                uint32_t *rclaim = &sh.claim[cstep % 3];
                ++cstep;
                resolve_expand_traces(s, sh, q, sh.ne, prune_on, amax, A.max_lag, rclaim);
                failed = __syncthreads_or(sh.err != 0);
            }
        }
        if (A.stats && threadIdx.x == 0) sh.st[1] += globaltimer_ns() - sh.t_phase;
        if (failed) break;
        if (sh.nq[d & 1] == 0) {
            status = P && A.max_lag > 0 ? GWFA_ERR_EMPTY_FRONTIER : GWFA_ERR_UNREACHABLE;
            break;
        }
        if constexpr (P) {
            if (A.evict_lag > 0 && d % A.evict_every == 0) {
                evict_behind(s, sh, amax, A.evict_lag, phase & 1, &sh.nq[d & 1]);
                failed = __syncthreads_or(sh.err != 0);
                if (failed) break;
            }
        }
    }
    __syncthreads();
    if (failed) status = sh.err;   // stable now: every thread has left the processing phases
    const uint32_t nt = sh.nt;
    if constexpr (!P) {
        // exact mode never removes a diagonal from H~, so the visited count is the
        // number of lanes of the touched tiles that hold an offset
        const uint32_t ntc = min(nt, s.cap);
        uint32_t c = 0;
        for (uint32_t t = threadIdx.x; t < ntc * kTile; t += blockDim.x)
            c += __ldcg(&s.slots[__ldcg(&s.touched[t / kTile])].vals[t % kTile]) >= 0 ? 1u : 0u;
        c = __reduce_add_sync(0xFFFFFFFFu, c);
        if ((threadIdx.x & 31) == 0 && c) atomicAdd(&sh.visited, (unsigned long long)c);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (status == GWFA_ERR_CAPACITY && A.retry) {
            const uint32_t r = atomicAdd(A.retry_count, 1u);
            A.retry[r] = qid;   // the retry list has room for every query
        } else {
            gwfa_result r = {};
            r.status = status;
            r.edit_distance = status == 0 ? d : -1;
            r.is_upper_bound = sh.pruned + sh.pruned32 > 0 ? 1 : 0;
            r.n_scores = (uint32_t)(d + 1);
            r.cells = sh.cells;
            r.visited = sh.visited + sh.visited32;
            r.peak_frontier = sh.peak;
            r.pruned = sh.pruned + sh.pruned32;
            r.spills = sh.spills + sh.spills32;
            r.evicted = sh.evicted;
            if constexpr (P) {
                if (A.traceback && status == 0) {
                    // GwfTraceback (Alg. 6): push the end vertex, then follow T back to the
                    // start and write the walk in order
                    const uint32_t te = push_trace(s, sh, (uint32_t)(sh.end_vp >> 32),
                                                   (uint32_t)sh.end_vp & 0xFFFFFFFFu);
                    uint32_t len = 0;
                    for (uint32_t t = te; t != kNoTrace && len <= sh.tlen; t = __ldcg(&s.trace[t]).y) ++len;
                    if (A.path_len) A.path_len[qid] = len;
                    uint32_t pos = len;
                    for (uint32_t t = te; t != kNoTrace && pos > 0; t = __ldcg(&s.trace[t]).y) {
                        --pos;
                        if (A.paths && pos < A.path_cap)
                            A.paths[(uint64_t)qid * A.path_cap + pos] = __ldcg(&s.trace[t]).x;
                    }
                }
            }
            r.device_us = (uint32_t)min((globaltimer_ns() - sh.t_start) / 1000ull, 0xFFFFFFFFull);
            A.out[qid] = r;
            if (A.stats) {
                unsigned long long *o = A.stats + (uint64_t)qid * kStatWords;
                for (int i = 0; i < 6; ++i) o[i] = sh.st[i];
                o[6] = sh.nt;
                o[7] = (unsigned long long)(d + 1);
            }
        }
    }
    wipe_touched<P>(s, nt);
    __syncthreads();
}

// The persistent loop of a CTA: pull a query id, run its score loop, repeat.
template <bool P>
__device__ __forceinline__ void align_queries(const TierArgs &A) {
    __shared__ Sh sh;
    // the slab's array pointers are the same for every thread: held once in shared
    // memory rather than in each thread's registers (where, at 32 registers, they
    // were spilled to local memory and reloaded through L1/L2 in the hot phases);
    // visible to all threads after the first barrier of the loop below
    __shared__ Slab<P> s;
    if (threadIdx.x == 0) s = carve<P>(A.slabs + (uint64_t)blockIdx.x * A.slab_bytes, A.log2cap);
    const uint32_t count = A.list_count ? *A.list_count : A.count_val;
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t t = atomicAdd(A.head, 1u);
            sh.qid = t < count ? (A.list ? A.list[A.list_offset + t] : A.list_offset + t) : 0xFFFFFFFFu;
        }
        __syncthreads();
        const uint32_t qid = sh.qid;
        __syncthreads();
        if (qid == 0xFFFFFFFFu) break;
        align_one<P>(A, s, sh, qid);
    }
}

// Up to 512 threads, 4 CTAs per SM at 32 registers: the throughput shape.
template <bool P>
__global__ void __launch_bounds__(512, 4) align_kernel(TierArgs A) {
    align_queries<P>(A);
}

// 1024 threads, 2 CTAs per SM at the same 32 registers: twice the groups on one
// query, for the few heaviest queries whose own latency bounds a batch.
template <bool P>
__global__ void __launch_bounds__(1024, 2) align_kernel_wide(TierArgs A) {
    align_queries<P>(A);
}

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Serving: a persistent kernel whose CTAs take requests from host-published rings
// (continuous batching: a CTA starts a new request as soon as it finishes one).
// CTAs [0, n_small) serve class 0 (small hash slabs), the rest class 1 (large
// slabs), which also take class-0 requests whenever no class-1 request waits, so
// large slabs are never left idle while small requests queue.  Every
// wait is bounded: a CTA idle for wait_limit polls votes idle (and withdraws the
// vote if work comes); the CTAs leave together once every CTA has voted, or after
// 16 x wait_limit polls in any case, and the host relaunches the kernel when work
// comes.  Leaving together keeps the full set of CTAs whenever the kernel runs.
template <bool P>
__global__ void __launch_bounds__(512, 4) server_kernel(ServerArgs S) {
    extern __shared__ uint32_t qsm[];   // the request's packed words, staged
    __shared__ Sh sh;
    __shared__ unsigned long long s_ticket;
    __shared__ uint64_t s_qoff[2];
    __shared__ uint32_t s_vs, s_ve;
    __shared__ int s_go, s_ring;
    const int cls = blockIdx.x < S.n_small ? 0 : 1;
    uint8_t *base = cls == 0 ? S.slabs + (uint64_t)blockIdx.x * S.slab_bytes[0]
                             : S.slabs + S.big_offset + (uint64_t)(blockIdx.x - S.n_small) * S.slab_bytes[1];
    __shared__ Slab<P> s;   // as in align_queries; visible after the first poll barrier
    if (threadIdx.x == 0) s = carve<P>(base, S.log2cap[cls]);
    for (;;) {
        if (threadIdx.x == 0) {
            int go = 0;
            uint32_t polls = 0;
            bool voted = false;
            for (;;) {
                if (ld_acquire_sys(S.stop)) break;
                // the CTA's own ring first; a large-slab CTA then looks at ring 0
                int rc = -1;
                unsigned long long h = 0;
                for (int c = cls; c >= 0; --c) {
                    const unsigned long long hc = atomicAdd(S.head + c, 0ull);
                    if (hc < ld_acquire_sys(S.tail[c])) {
                        rc = c;
                        h = hc;
                        break;
                    }
                }
                if (rc >= 0) {
                    if (voted) {
                        atomicSub(S.idle_votes, 1u);
                        voted = false;
                    }
                    polls = 0;
                    if (atomicCAS(S.head + rc, h, h + 1) == h) {
                        s_ticket = h;
                        s_ring = rc;
                        go = 1;
                        break;
                    }
                    continue;
                }
                ++polls;
                if (!voted && polls > S.wait_limit) {
                    atomicAdd(S.idle_votes, 1u);
                    voted = true;
                }
                if (voted && (atomicAdd(S.idle_votes, 0u) >= S.n_ctas || polls > 16u * S.wait_limit)) {
                    atomicAdd(S.timeouts, 1ull);
                    break;
                }
                __nanosleep(S.sleep_ns);
            }
            s_go = go;
        }
        __syncthreads();
        if (!s_go) break;
        const unsigned long long ticket = s_ticket;
        const int rc = s_ring;   // the ring the request came from (its result goes back there)
        const uint32_t slot = (uint32_t)(ticket % S.ring);
        const ReqDesc *d = S.desc[rc] + slot;
        const uint32_t n = __ldcv(&d->n);
        const uint32_t nw = (n + 15) >> 4;
        const uint32_t *src = S.arena[rc] + (uint64_t)slot * S.slot_words;
        for (uint32_t w = threadIdx.x; w < nw + 2; w += blockDim.x) qsm[w] = w < nw ? __ldcv(src + w) : 0u;
        if (threadIdx.x == 0) {
            s_qoff[0] = 0;
            s_qoff[1] = n;
            s_vs = __ldcv(&d->v_s);
            s_ve = __ldcv(&d->v_e);
        }
        __syncthreads();
        TierArgs A{};
        A.g = S.g;
        A.qwords = qsm;
        A.q_smem = 1;
        A.q_off = s_qoff;
        A.v_s = &s_vs;
        A.v_e = &s_ve;
        A.out = S.results[rc] + slot;
        A.max_lag = S.max_lag;
        A.max_score = S.max_score;
        align_one<P>(A, s, sh, 0);
        if (threadIdx.x == 0) {
            __threadfence_system();
            st_release_sys(S.done[rc] + slot, ticket + 1);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int base_code(unsigned char c) {
    switch (c) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    default: return -1;
    }
}

// 2-bit packing of the queries (a2): one warp per query, one 16-base word per lane.
__global__ void pack_kernel(uint32_t nq, const char *__restrict__ q, const uint64_t *__restrict__ off,
                            uint32_t *__restrict__ words, int32_t *__restrict__ status) {
    const int lane = threadIdx.x & 31;
    const uint32_t wpb = blockDim.x >> 5;
    for (uint32_t qi = blockIdx.x * wpb + (threadIdx.x >> 5); qi < nq; qi += gridDim.x * wpb) {
        const uint64_t a = off[qi], n = off[qi + 1] - a;
        const uint64_t w0 = (a >> 4) + qi, nw = (n + 15) >> 4;
        bool bad = false;
        for (uint64_t t = lane; t < nw; t += 32) {
            uint32_t w = 0;
            for (int c = 0; c < 16; ++c) {
                const uint64_t p = t * 16 + c;
                if (p < n) {
                    int code = base_code((unsigned char)q[a + p]);
                    if (code < 0) { bad = true; code = 0; }
                    w |= (uint32_t)code << (2 * c);
                }
            }
            words[w0 + t] = w;
        }
        bad = __any_sync(0xFFFFFFFFu, bad);
        if (lane == 0 && status) status[qi] = bad ? GWFA_ERR_INVALID : 0;
    }
    if (blockIdx.x == 0 && threadIdx.x < 2) words[(off[nq] >> 4) + nq + threadIdx.x] = 0;
}

__global__ void fill_kernel(uint4 *p, uint64_t n16) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n16;
         i += (uint64_t)gridDim.x * blockDim.x)
        p[i] = make_uint4(~0u, ~0u, ~0u, ~0u);
}

// Slabs start empty: slot keys and offsets all ones (empty / absent), lane-mask
// words 0 (the second 8 bytes of every slot).  Only the hash slots are written:
// every list of the slab (touched, Q, spills, frontier snapshots, spill requests,
// T) is written before it is read.
__global__ void slab_init_kernel(uint8_t *slabs, uint64_t slab_bytes, uint32_t n_slabs,
                                 uint64_t slots_bytes, uint64_t slot_bytes) {
    const uint64_t per = slots_bytes / 16, total = per * n_slabs;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t o = (i % per) * 16;   // offset inside the slab's slot region
        uint4 *p = (uint4 *)(slabs + (i / per) * slab_bytes + o);
        *p = o % slot_bytes == 0 ? make_uint4(~0u, ~0u, 0u, 0u) : make_uint4(~0u, ~0u, ~0u, ~0u);
    }
}

}  // namespace

cudaError_t launch_align(const TierArgs &a, bool prune, uint32_t ctas, uint32_t threads,
                         cudaStream_t st) {
    if (threads > 512) {
        if (prune) align_kernel_wide<true><<<ctas, threads, 0, st>>>(a);
        else align_kernel_wide<false><<<ctas, threads, 0, st>>>(a);
    } else {
        if (prune) align_kernel<true><<<ctas, threads, 0, st>>>(a);
        else align_kernel<false><<<ctas, threads, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_server(const ServerArgs &a, bool prune, uint32_t ctas, uint32_t threads,
                          uint32_t smem_bytes, cudaStream_t st) {
    if (prune) {
        cudaFuncSetAttribute(server_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
        server_kernel<true><<<ctas, threads, smem_bytes, st>>>(a);
    } else {
        cudaFuncSetAttribute(server_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
        server_kernel<false><<<ctas, threads, smem_bytes, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_pack(uint32_t nq, const char *d_q, const uint64_t *d_off, uint32_t *d_words,
                        int32_t *d_status, cudaStream_t st) {
    uint32_t blocks = (nq + 7) / 8;
    if (blocks == 0) blocks = 1;
    if (blocks > 65535) blocks = 65535;
    pack_kernel<<<blocks, 256, 0, st>>>(nq, d_q, d_off, d_words, d_status);
    return cudaGetLastError();
}

cudaError_t launch_fill(void *p, uint64_t bytes, cudaStream_t st) {
    const uint64_t n16 = bytes / 16;
    if (n16 == 0) return cudaSuccess;
    uint64_t blocks = (n16 + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    fill_kernel<<<(unsigned)blocks, 256, 0, st>>>((uint4 *)p, n16);
    return cudaGetLastError();
}

cudaError_t launch_slab_init(uint8_t *slabs, uint64_t slab_bytes, uint32_t n_slabs, uint32_t log2cap,
                             bool prune, cudaStream_t st) {
    const SlabLayout L = slab_layout(log2cap, prune);
    const uint64_t n16 = (L.touched - L.slots) / 16 * n_slabs;
    if (n16 == 0) return cudaSuccess;
    uint64_t blocks = (n16 + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    slab_init_kernel<<<(unsigned)blocks, 256, 0, st>>>(slabs, slab_bytes, n_slabs,
                                                        L.touched - L.slots, L.slot_bytes);
    return cudaGetLastError();
}

// Load the alignment kernels into the context now.  With lazy module loading a
// kernel's code is loaded at its first launch, and that load can wait for kernels
// already running; an engine runs several of them side by side (its classes
// beside tier 0), so it touches them all before the first one starts.
cudaError_t preload_kernels() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, align_kernel<false>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, align_kernel<true>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, align_kernel_wide<false>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, align_kernel_wide<true>);
    return e;
}

int align_occupancy(bool prune, uint32_t threads, int *blocks_per_sm) {
    cudaError_t e = prune
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, align_kernel<true>, (int)threads, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, align_kernel<false>, (int)threads, 0);
    return e == cudaSuccess ? 0 : -1;
}

}  // namespace gwfa
