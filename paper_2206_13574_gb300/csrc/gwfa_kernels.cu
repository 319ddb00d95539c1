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
//   reg    two words per tile, used alternately by successive phases:
//          (phase stamp << 32 | lane mask).  The first lane to register a tile in
//          a phase appends the tile to that phase's list, so every list holds a
//          tile once, with the mask of its live diagonals.
//   Q      qlist: tiles live after GwfExpand (the queue Q of Alg. 1-3).
//   spill  slist[2]: tiles that received offset 0 by a spill in the current
//          extension round; they are extended in the same score (Alg. 2 pushes
//          them onto the queue being drained).
//   E      the extended frontier (Q' of Alg. 2): tile, mask and a snapshot of the
//          8 offsets after extension.  GwfExpand reads the snapshot, so its
//          sources are the offsets before any of its own writes (the H~ / H~'
//          split of Alg. 3) and it can max-merge straight into H~ with atomics.
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
    unsigned long long *keys;
    unsigned long long *reg[2];
    T *vals;
    uint32_t *touched, *qlist, *slist[2], *eslot, *emask;
    T *evals;
    int4 *req;
    uint32_t cap, mask;
};

template <bool P>
__device__ __forceinline__ Slab<P> carve(uint8_t *base, uint32_t log2cap) {
    SlabLayout L = slab_layout(log2cap, P);
    Slab<P> s;
    s.keys = (unsigned long long *)(base + L.keys);
    s.reg[0] = (unsigned long long *)(base + L.reg0);
    s.reg[1] = (unsigned long long *)(base + L.reg1);
    s.vals = (typename VT<P>::T *)(base + L.vals);
    s.touched = (uint32_t *)(base + L.touched);
    s.qlist = (uint32_t *)(base + L.qlist);
    s.slist[0] = (uint32_t *)(base + L.slist0);
    s.slist[1] = (uint32_t *)(base + L.slist1);
    s.eslot = (uint32_t *)(base + L.eslot);
    s.emask = (uint32_t *)(base + L.emask);
    s.evals = (typename VT<P>::T *)(base + L.evals);
    s.req = (int4 *)(base + L.req);
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
    uint32_t nreq[2];   // pending spill requests (pruning mode), by generation parity
    uint32_t ne;        // extended-frontier entries this score
    uint32_t nt;        // tiles claimed (touched) this query
    uint32_t score_cells;
    unsigned long long amax;
    unsigned long long cells, visited, pruned, spills;
    uint32_t peak;
};

__device__ __forceinline__ void set_err(Sh &sh, int code) { atomicCAS(&sh.err, 0, code); }

// 16 bases starting at base position p of a packed stream.
__device__ __forceinline__ uint32_t window16(const uint32_t *__restrict__ w, uint64_t p) {
    const uint64_t wi = p >> 4;
    const uint32_t sh = (uint32_t)(p & 15) * 2;
    const uint32_t lo = __ldg(w + wi), hi = __ldg(w + wi + 1);
    return __funnelshift_r(lo, hi, sh);
}

// LCP(q[i+1..|q|], v[j+1..|v|]) of Eq. 2 in 0-based positions: XOR of 16-base
// windows, the first differing base is the lowest set bit pair.
__device__ __forceinline__ int lcp(const uint32_t *__restrict__ qw, int i, int n,
                                   const uint32_t *__restrict__ vw, int j, int lv) {
    const int maxl = min(n - i, lv - j);
    int l = 0;
    while (l < maxl) {
        const uint32_t x = window16(qw, (uint64_t)(i + l)) ^ window16(vw, (uint64_t)(j + l));
        if (x) {
            l += (__ffs(x) - 1) >> 1;
            break;
        }
        l += 16;
    }
    return min(l, maxl);
}

__device__ __forceinline__ unsigned long long tile_key(uint32_t v, int kb) {
    return ((unsigned long long)v << 32) | (uint32_t)kb;
}

template <bool P>
__device__ int find_or_insert(const Slab<P> &s, Sh &sh, unsigned long long key) {
    uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 32) & s.mask;
    for (int probe = 0; probe < 256; ++probe) {
        const unsigned long long cur = __ldcg(&s.keys[h]);
        if (cur == key) return (int)h;
        if (cur == kEmptyKey) {
            const unsigned long long prev = atomicCAS(&s.keys[h], kEmptyKey, key);
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

// Register lane `bit` of a tile for phase `stamp`; true for the first lane of the
// tile in this phase (that caller appends the tile to the phase's list).
__device__ __forceinline__ bool reg_lane(unsigned long long *w, uint32_t stamp, uint32_t bit,
                                         Sh &sh) {
    unsigned long long old = __ldcg(w);
    for (int it = 0; it < 64; ++it) {
        if ((uint32_t)(old >> 32) == stamp) {
            atomicOr(w, (unsigned long long)bit);
            return false;
        }
        const unsigned long long nw = ((unsigned long long)stamp << 32) | bit;
        const unsigned long long prev = atomicCAS(w, old, nw);
        if (prev == old) return true;
        old = prev;
    }
    set_err(sh, GWFA_ERR_CAPACITY);
    return false;
}

__device__ __forceinline__ void list_append(uint32_t *list, uint32_t *count, uint32_t cap,
                                            uint32_t slot, Sh &sh) {
    const uint32_t i = atomicAdd(count, 1u);
    if (i < cap) list[i] = slot;
    else set_err(sh, GWFA_ERR_CAPACITY);
}

struct QCtx {
    const uint32_t *qw;   // this query's packed words
    int n;
    uint32_t ve;
    int ke;
    uint32_t lve;
};

// Offer value `cand` to diagonal lane `ln` of tile `slot` (GwfExpand's max-merge
// into H~); registers the lane in the next Q if its offset strictly improved.
template <bool P>
__device__ __forceinline__ void offer(const Slab<P> &s, Sh &sh, int slot, int ln,
                                      typename VT<P>::T cand, uint32_t stamp, int par,
                                      uint32_t *qcount) {
    const typename VT<P>::T prev = atomicMax(&s.vals[(uint32_t)slot * kTile + ln], cand);
    if (prev < 0) atomicAdd(&sh.visited, 1ull);
    if (pj(prev) < pj(cand)) {
        if (reg_lane(&s.reg[par][slot], stamp, 1u << ln, sh))
            list_append(s.qlist, qcount, s.cap, (uint32_t)slot, sh);
    }
}

// Spill of Alg. 2: diagonal (v, k) reached |v|; offset 0 (with walk base
// `base + |v|`) goes to (u, k + |v|) for every arc (v, u) where it is absent.
template <bool P>
__device__ void spill_arcs(const DevGraph &g, const Slab<P> &s, Sh &sh, uint32_t v, int k,
                           uint32_t lv, uint32_t base, uint32_t stamp, int par,
                           uint32_t *next_list, uint32_t *next_count) {
    const uint32_t a0 = __ldg(&g.arc_off[v]), a1 = __ldg(&g.arc_off[v + 1]);
    const int ku = k + (int)lv;
    const uint32_t nb = base + lv;
    if (P && nb > kBaseMask) { set_err(sh, GWFA_ERR_CAPACITY); return; }
    for (uint32_t a = a0; a < a1; ++a) {
        const uint32_t u = __ldg(&g.arc_dst[a]);
        const int su = find_or_insert(s, sh, tile_key(u, ku >> 3));
        if (su < 0) return;
        const int ln = ku & 7;
        typename VT<P>::T cand;
        if constexpr (P) cand = pk(0, kTagPend, nb);
        else cand = 0;
        const typename VT<P>::T prev = atomicMax(&s.vals[(uint32_t)su * kTile + ln], cand);
        if (prev < 0) {
            atomicAdd(&sh.visited, 1ull);
            atomicAdd(&sh.spills, 1ull);
            if (reg_lane(&s.reg[par][su], stamp, 1u << ln, sh))
                list_append(next_list, next_count, s.cap, (uint32_t)su, sh);
        }
    }
}

// One extension round over `list` (tiles registered at phase `cur_stamp`).
template <bool P>
__device__ void extend_round(const DevGraph &g, const Slab<P> &s, Sh &sh, const QCtx &q,
                             const uint32_t *list, uint32_t n_list, int cur_par,
                             uint32_t next_stamp, int next_par, uint32_t *next_list,
                             uint32_t *next_count, uint32_t *req_count) {
    using T = typename VT<P>::T;
    const int gid = threadIdx.x >> 3, ln = threadIdx.x & 7, ngroups = blockDim.x >> 3;
    const unsigned gmask = 0xFFu << (threadIdx.x & 24);
    for (uint32_t e = gid; e < n_list; e += ngroups) {
        const uint32_t slot = __ldcg(&list[e]);
        const unsigned long long key = __ldcg(&s.keys[slot]);
        const uint32_t m = (uint32_t)__ldcg(&s.reg[cur_par][slot]) & 0xFFu;
        const uint32_t v = (uint32_t)(key >> 32);
        const int k = (int)(uint32_t)key * kTile + ln;
        uint32_t eidx = 0;
        if (ln == 0) {
            eidx = atomicAdd(&sh.ne, 1u);
            atomicAdd(&sh.score_cells, (uint32_t)__popc(m));
        }
        eidx = __shfl_sync(gmask, eidx, 0, 8);
        T val = (T)-1;
        unsigned long long a = 0;
        if ((m >> ln) & 1u) {
            val = __ldcg(&s.vals[slot * kTile + ln]);
            const int j = pj(val);
            const uint32_t lv = __ldg(&g.vlen[v]);
            const int i = k + j;
            const int l = lcp(q.qw, i, q.n, g.words + __ldg(&g.vstart[v]), j, (int)lv);
            const int j2 = j + l;
            if constexpr (P) val = pk(j2, kTagSettled, pbase(val));
            else val = j2;
            __stcg(&s.vals[slot * kTile + ln], val);
            if (v == q.ve && k == q.ke && (uint32_t)j2 == lv) sh.found = 1;
            if constexpr (P) a = (unsigned long long)(long long)(i + l) + pbase(val) + (unsigned)j2;
            if ((uint32_t)j2 == lv) {
                if constexpr (P) {
                    const uint32_t r = atomicAdd(req_count, 1u);
                    if (r < s.cap) s.req[r] = make_int4((int)v, k, (int)pbase(val), (int)lv);
                    else set_err(sh, GWFA_ERR_CAPACITY);
                } else {
                    spill_arcs<P>(g, s, sh, v, k, lv, 0u, next_stamp, next_par, next_list,
                                  next_count);
                }
            }
        }
        if constexpr (P) {
            // a = i + W~ of Alg. 4, reduced over the tile then the CTA
            for (int o = 4; o >= 1; o >>= 1) {
                const unsigned long long b = __shfl_xor_sync(gmask, a, o, 8);
                a = b > a ? b : a;
            }
            if (ln == 0 && a > 0) atomicMax(&sh.amax, a);
        }
        if (eidx < s.cap) {
            if (ln == 0) {
                __stcg(&s.eslot[eidx], slot);
                __stcg(&s.emask[eidx], m);
            }
            __stcg(&s.evals[eidx * kTile + ln], val);
        } else if (ln == 0) {
            set_err(sh, GWFA_ERR_CAPACITY);
        }
    }
}

// Pruning mode, second half of a round: apply the recorded spills after every
// diagonal of the round has been extended, so that a spill can never touch a
// diagonal that was present before the round (Alg. 2's presence test).
__device__ void apply_spill_requests(const DevGraph &g, const Slab<true> &s, Sh &sh,
                                     uint32_t n_req, uint32_t stamp, int par,
                                     uint32_t *next_list, uint32_t *next_count) {
    const uint32_t nr = min(n_req, s.cap);
    for (uint32_t r = threadIdx.x; r < nr; r += blockDim.x) {
        const int4 q = __ldcg(&s.req[r]);
        spill_arcs<true>(g, s, sh, (uint32_t)q.x, q.y, (uint32_t)q.w, (uint32_t)q.z, stamp, par,
                         next_list, next_count);
    }
}

// GwfExpand (Alg. 3) over the extended frontier, with GwfPrune (Alg. 4) applied
// to the sources on the way in.
template <bool P>
__device__ void expand_all(const DevGraph &g, const Slab<P> &s, Sh &sh, const QCtx &q,
                           uint32_t n_e, bool prune_on, long long amax, int max_lag,
                           uint32_t stamp, int par, uint32_t *qcount) {
    using T = typename VT<P>::T;
    const int gid = threadIdx.x >> 3, ln = threadIdx.x & 7, ngroups = blockDim.x >> 3;
    const uint32_t ne = min(n_e, s.cap);
    // warp-uniform trip count: every lane of a warp reaches the shuffles together
    for (uint32_t base = 0; base < ne; base += ngroups) {
        const uint32_t e = base + gid;
        const bool valid = e < ne;
        uint32_t slot = 0, m = 0, v = 0, lv = 0;
        int kb = 0;
        T val = (T)-1;
        if (valid) {
            slot = __ldcg(&s.eslot[e]);
            m = __ldcg(&s.emask[e]);
            val = __ldcg(&s.evals[e * kTile + ln]);
            const unsigned long long key = __ldcg(&s.keys[slot]);
            v = (uint32_t)(key >> 32);
            kb = (int)(uint32_t)key;
            lv = __ldg(&g.vlen[v]);
        }
        bool act = valid && ((m >> ln) & 1u);
        const int k = kb * kTile + ln;
        const int j = act ? pj(val) : 0;
        const int i = k + j;
        const uint32_t b = pbase(val);
        if (P && act && prune_on) {
            const long long a = (long long)i + (long long)b + j;
            if (amax - a >= (long long)max_lag) {
                act = false;
                atomicAdd(&sh.pruned, 1ull);
            }
        }
        const bool ins = act && i < q.n;            // (k+1, j)
        const bool del = act && j < (int)lv;        // (k-1, j+1)
        const bool mis = ins && j < (int)lv;        // (k, j+1)
        T c_ins, c_del, c_mis;
        if constexpr (P) {
            c_ins = ins ? pk(j, kTagFresh, b) : -1ll;
            c_del = del ? pk(j + 1, kTagFresh, b) : -1ll;
            c_mis = mis ? pk(j + 1, kTagFresh, b) : -1ll;
        } else {
            c_ins = ins ? j : -1;
            c_del = del ? j + 1 : -1;
            c_mis = mis ? j + 1 : -1;
        }
        T from_left = __shfl_up_sync(0xFFFFFFFFu, c_ins, 1, 8);
        T from_right = __shfl_down_sync(0xFFFFFFFFu, c_del, 1, 8);
        if (ln == 0) from_left = (T)-1;
        if (ln == 7) from_right = (T)-1;
        T cand = c_mis;
        if (from_left > cand) cand = from_left;
        if (from_right > cand) cand = from_right;
        if (valid && cand >= 0) offer<P>(s, sh, (int)slot, ln, cand, stamp, par, qcount);
        if (valid && ln == 7 && ins) {   // insertion leaves the tile: (v, 8(kb+1))
            const int t = find_or_insert(s, sh, tile_key(v, kb + 1));
            if (t >= 0) offer<P>(s, sh, t, 0, c_ins, stamp, par, qcount);
        }
        if (valid && ln == 0 && del) {   // deletion leaves the tile: (v, 8 kb - 1)
            const int t = find_or_insert(s, sh, tile_key(v, kb - 1));
            if (t >= 0) offer<P>(s, sh, t, 7, c_del, stamp, par, qcount);
        }
    }
}

template <bool P>
__device__ void wipe_touched(const Slab<P> &s, uint32_t nt) {
    using T = typename VT<P>::T;
    nt = min(nt, s.cap);
    for (uint32_t t = threadIdx.x; t < nt * kTile; t += blockDim.x) {
        const uint32_t slot = __ldcg(&s.touched[t / kTile]);
        __stcg(&s.vals[slot * kTile + (t % kTile)], (T)-1);
        if (t % kTile == 0) {
            __stcg(&s.keys[slot], kEmptyKey);
            __stcg(&s.reg[0][slot], ~0ull);
            __stcg(&s.reg[1][slot], ~0ull);
        }
    }
}

template <bool P>
__device__ void align_one(const TierArgs &A, const Slab<P> &s, Sh &sh, uint32_t qid) {
    const DevGraph &g = A.g;
    const uint64_t qo = A.q_off[qid];
    const int n = (int)(A.q_off[qid + 1] - qo);
    QCtx q;
    q.qw = A.qwords + (qo >> 4) + qid;
    q.n = n;
    const uint32_t vs = A.v_s[qid];
    q.ve = A.v_e[qid];
    int pre = 0;
    if (A.qstatus) pre = A.qstatus[qid];
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
    q.lve = __ldg(&g.vlen[q.ve]);
    q.ke = n - (int)q.lve;

    // Alg. 1 initialisation: H~_{v_s,0} <- 0, Q <- [(v_s, 0)], d <- 0
    if (threadIdx.x == 0) {
        sh.err = 0;
        sh.nt = 0;
        sh.cells = sh.visited = sh.pruned = sh.spills = 0;
        sh.peak = 0;
        sh.nq[0] = sh.nq[1] = 0;
        const int slot = find_or_insert(s, sh, tile_key(vs, 0));
        if (slot >= 0) {
            typename VT<P>::T v0;
            if constexpr (P) v0 = pk(0, kTagFresh, 0);
            else v0 = 0;
            s.vals[(uint32_t)slot * kTile] = v0;
            sh.visited = 1;
            reg_lane(&s.reg[1][slot], 1u, 1u, sh);
            s.qlist[0] = (uint32_t)slot;
            sh.nq[0] = 1;
        }
    }
    __syncthreads();

    uint32_t stamp = 1;   // phase stamp of the tiles in Q
    int d = 0;
    int status = 0;
    int failed = 0;
    for (;;) {
        // ---- GwfExtend (Alg. 2), one breadth-first round per loop iteration
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
        const uint32_t *list = s.qlist;
        uint32_t n_list = min(sh.nq[d & 1], s.cap);
        for (int gen = 0;; ++gen) {
            const uint32_t next_stamp = stamp + 1;
            uint32_t *next_list = s.slist[(gen + 1) & 1];
            // round g fills ns[(g+1)%3] and clears ns[(g+2)%3] for round g+1; the
            // cleared counter was last read before the previous round's barrier
            uint32_t *next_count = &sh.ns[(gen + 1) % 3];
            if (threadIdx.x == 0) sh.ns[(gen + 2) % 3] = 0;
            extend_round<P>(g, s, sh, q, list, n_list, stamp & 1, next_stamp, next_stamp & 1,
                            next_list, next_count, &sh.nreq[gen & 1]);
            if constexpr (P) {
                __syncthreads();
                if (threadIdx.x == 0) sh.nreq[(gen + 1) & 1] = 0;
                apply_spill_requests(g, s, sh, sh.nreq[gen & 1], next_stamp, next_stamp & 1,
                                     next_list, next_count);
            }
            // every exit decision comes from a barrier reduction: sh.err may be set by
            // threads that already run the next phase, so it is never re-read for control
            failed = __syncthreads_or(sh.err != 0);
            const uint32_t ns = *next_count;
            stamp = next_stamp;
            if (failed || ns == 0) break;
            list = next_list;
            n_list = min(ns, s.cap);
        }
        if (threadIdx.x == 0) {
            sh.cells += sh.score_cells;
            sh.peak = max(sh.peak, sh.score_cells);
        }
        if (failed) break;
        // end test of Alg. 1
        if (sh.found) break;
        if (A.max_score >= 0 && d >= A.max_score) { status = GWFA_ERR_SCORE_LIMIT; break; }
        d = d + 1;
        // ---- GwfPrune (Alg. 4) folded into the sources of GwfExpand (Alg. 3)
        const long long amax = (long long)sh.amax;
        const bool prune_on = P && A.max_lag > 0 && amax > (long long)A.max_lag;
        stamp = stamp + 1;
        expand_all<P>(g, s, sh, q, sh.ne, prune_on, amax, A.max_lag, stamp, stamp & 1,
                      &sh.nq[d & 1]);
        failed = __syncthreads_or(sh.err != 0);
        if (failed) break;
        if (sh.nq[d & 1] == 0) {
            status = P && A.max_lag > 0 ? GWFA_ERR_EMPTY_FRONTIER : GWFA_ERR_UNREACHABLE;
            break;
        }
        if (stamp > 0xF0000000u) { status = GWFA_ERR_CAPACITY; break; }
    }
    __syncthreads();
    if (failed) status = sh.err;   // stable now: every thread has left the processing phases
    const uint32_t nt = sh.nt;
    if (threadIdx.x == 0) {
        if (status == GWFA_ERR_CAPACITY && A.retry) {
            const uint32_t r = atomicAdd(A.retry_count, 1u);
            A.retry[r] = qid;   // the retry list has room for every query
        } else {
            gwfa_result r = {};
            r.status = status;
            r.edit_distance = status == 0 ? d : -1;
            r.is_upper_bound = sh.pruned > 0 ? 1 : 0;
            r.n_scores = (uint32_t)(d + 1);
            r.cells = sh.cells;
            r.visited = sh.visited;
            r.peak_frontier = sh.peak;
            r.pruned = sh.pruned;
            r.spills = sh.spills;
            A.out[qid] = r;
        }
    }
    wipe_touched<P>(s, nt);
    __syncthreads();
}

template <bool P>
__global__ void __launch_bounds__(512) align_kernel(TierArgs A) {
    __shared__ Sh sh;
    const Slab<P> s = carve<P>(A.slabs + (uint64_t)blockIdx.x * A.slab_bytes, A.log2cap);
    const uint32_t count = A.list_count ? *A.list_count : A.count_val;
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t t = atomicAdd(A.head, 1u);
            sh.qid = t < count ? (A.list ? A.list[t] : t) : 0xFFFFFFFFu;
        }
        __syncthreads();
        const uint32_t qid = sh.qid;
        __syncthreads();
        if (qid == 0xFFFFFFFFu) break;
        align_one<P>(A, s, sh, qid);
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

}  // namespace

cudaError_t launch_align(const TierArgs &a, bool prune, uint32_t ctas, uint32_t threads,
                         cudaStream_t st) {
    if (prune) align_kernel<true><<<ctas, threads, 0, st>>>(a);
    else align_kernel<false><<<ctas, threads, 0, st>>>(a);
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

int align_occupancy(bool prune, uint32_t threads, int *blocks_per_sm) {
    cudaError_t e = prune
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, align_kernel<true>, (int)threads, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, align_kernel<false>, (int)threads, 0);
    return e == cudaSuccess ? 0 : -1;
}

}  // namespace gwfa
