// ann_search_dev.cuh -- device code of Algorithm 1 (Sec. 4.2) of arXiv:1312.3062
// on sm_103a, shared by the translation units that instantiate its kernels.
//
// One warp runs one query from start to finish:
//   1. part tables  D_p[c] = ||q^p - c_p||^2           (Sec. 4.2, first step)
//   2. per-part sort by (key, center id) -> ranks        (Sec. 4.2)
//   3. the main loop of Algorithm 1: a shared min-queue of reference vectors
//      and the current bridge vector, the visited set (Color), the result set
//      R and the exact budget T.
// Bridge vectors are produced in the order of the multi-sequence algorithm
// (Sec. 3.3): ascending (bridge key, rank tuple).  A popped bridge vector
// with an empty list discovers nothing and only makes the next one current,
// so Algorithm 1's result depends only on the order of the NON-EMPTY bridges.
// The GPU therefore generates exactly that subsequence, in batches: a walk of
// the prefix index of non-empty bridges emits every bridge whose
// (key, ranks) lies in a window (lo, hi], and the batch is sorted.  The
// window grows geometrically; an overfull window is halved.
//
// All per-query state lives in the warp's slice of shared memory; no device
// trap or unbounded wait exists on this path.  Keys are squared distances:
// exact uint32 for uint8 data; for float32 data the float32 nearest to the
// exact value (double-float accumulation, then one rounding).  A float32
// bridge key is the float32 nearest to the exact sum of its float32 part
// keys; the walk skips work only on bounds taken with directed rounding.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <vector>

#include "ann_device.cuh"
#include "ann_internal.cuh"

namespace ann {

// ---------------------------------------------------------------------------
// shared-memory layout of one warp
// ---------------------------------------------------------------------------
struct WarpLayout {
    uint32_t q, tabD, rank, sk, sc, heap, hash, rbuf, bkey, bidx, pref, nodes, cand, ckey, wref, wkey, stage, misc,
        total;
    uint32_t heap_cap, hash_log, bcap, ncap, gcap, glist, stage_rows, stage_stride;
    uint32_t sc_parts;  // parts whose centers are kept in rank order (all of them when split walks may run)
};

// Rows of the next pop's neighbours staged in shared memory: on when a whole
// adjacency list of vectors fits in this many bytes.
constexpr uint32_t kStageBytes = 4096;

// Large-budget ("spilling") kernels keep at most this many queue entries in
// shared memory by default (the autotuner also tries other capacities); the
// rest of the queue and the visited set live in the warp's global scratch,
// so a query's shared-memory slice does not grow with the budget.
constexpr uint32_t kSpillHeap = 512;

__host__ __device__ inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline WarpLayout make_layout(int dtype, int d, int P, int n, int PA, int capT,
                                                  int kmax, int bcap, int b, int R, bool stage = true,
                                                  bool grouped = false, bool spill = false,
                                                  uint32_t spill_heap = kSpillHeap) {
    WarpLayout L;
    uint32_t o = 0;
    L.q = o;      o = align_up(o + (uint32_t)d * (dtype == ANN_U8 ? 1u : 4u), 16);
    L.tabD = o;   o = align_up(o + 4u * P * n, 16);
    L.rank = o;   o = align_up(o + (uint32_t)P * n, 16);
    L.sk = 0;     // sorted keys are read as D[sc[r]]
    // center id at each rank: the prefix parts, and with the large-budget
    // layout every part (the suffix pass of a split walk reads them); below
    // it the extra bytes would cost a resident query per SM
    L.sc_parts = spill ? (uint32_t)P : (uint32_t)PA;
    L.sc = o;     o = align_up(o + L.sc_parts * n, 16);
    uint32_t lpn = 1;
    while (lpn < (uint32_t)n) lpn <<= 1;  // the per-part sort borrows the heap region
    const uint32_t qcap = spill && (uint32_t)capT > spill_heap ? spill_heap : (uint32_t)capT;
    uint32_t hc = qcap > lpn ? qcap : lpn;
    L.heap_cap = hc;
    L.heap = o;   o = align_up(o + 8u * hc, 16);
    uint32_t hl = 5;
    while ((1u << hl) < 2u * (uint32_t)capT) hl++;
    L.hash_log = hl;
    L.hash = o;   o = align_up(o + (spill ? 0u : 4u * (1u << hl)), 16);  // spilling: in global scratch
    L.rbuf = o;   o = align_up(o + 8u * kmax, 16);
    L.bcap = (uint32_t)bcap;
    L.bkey = o;   o = align_up(o + 8u * bcap, 16);
    L.bidx = o;   o = align_up(o + 4u * bcap, 16);
    // candidate ids + keys of the main loop
    const uint32_t wb = 32u * (uint32_t)b;  // bridge-window entries
    uint32_t cand_n = wb > 32u ? wb : 32u;
    L.cand = o;   o = align_up(o + 4u * cand_n, 16);
    L.ckey = o;   o = align_up(o + 4u * cand_n, 16);
    // one region shared by three users that are never live at the same time:
    // the walk (prefix sums + node list), the bridge window (reference ids +
    // keys) and the staged neighbour vectors of the next pop
    const uint32_t vb = (uint32_t)d * (dtype == ANN_U8 ? 1u : 4u);
    L.stage_rows = stage && (uint32_t)R * vb <= kStageBytes ? (uint32_t)R : 0u;
    // walk lists: prefix nodes (4 words each) and, with the group level, c2
    // groups (5 words each)
    L.ncap = grouped ? 32 : 64;
    L.gcap = grouped ? 48 : 0;
    const uint32_t walk_bytes = align_up(4u * (n + 1), 16) + 16u * L.ncap + 20u * L.gcap;
    const uint32_t win_bytes = 2u * align_up(4u * wb, 16);
    // staged rows are padded by 16 bytes so that lanes reading different rows
    // at the same offset fall into different banks
    L.stage_stride = vb + 16;
    const uint32_t stage_bytes = L.stage_rows * L.stage_stride;
    uint32_t ub = walk_bytes > win_bytes ? walk_bytes : win_bytes;
    if (stage_bytes > ub) ub = stage_bytes;
    L.pref = o;
    L.nodes = o + align_up(4u * (n + 1), 16);
    L.glist = L.nodes + 16u * L.ncap;
    L.wref = o;
    L.wkey = o + align_up(4u * wb, 16);
    L.stage = o;
    o = align_up(o + ub, 16);
    L.misc = o;   o = align_up(o + 16u * 4, 16);  // [0] emit count, [3] min suffix, [4] min last part, [8..10] walk counters
    L.total = o;
    return L;
}

struct SearchArgs {
    DevIndex ix;
    const void *queries;
    int64_t nq;
    const int32_t *k;
    const int32_t *T;
    int32_t k_all, T_all, kmax;
    int32_t *out_ids;
    void *out_keys;
    int32_t *out_status;
    int64_t *out_stats;
    // query selection: list (nullable) of query indices; count from *list_count if non-null
    const int32_t *list;
    const int32_t *list_count;
    int64_t list_len;
    // persistent mode: work ticket counter (nullable)
    int32_t *ticket;
    int capT;
    int bcap;
    WarpLayout L;
    // per-warp global scratch of the large-budget kernels, wstride bytes per
    // warp: sorted bridge windows (gcap x (2 keys + 2 values)) at 0, the
    // queue's overflow (capT entries) at spill_off, the visited set
    // (2^hash_log slots) at hash_off
    uint8_t *gscratch;
    uint32_t gcap;
    uint64_t wstride, spill_off, hash_off;
};

// ---------------------------------------------------------------------------
// visited set: open addressing over ids (slot = id + 1, 0 = empty)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t hslot(uint32_t x, uint32_t log) {
    return (x * 2654435761u) >> (32 - log);
}
__device__ __forceinline__ bool hash_has(const uint32_t *H, uint32_t log, uint32_t x) {
    uint32_t mask = (1u << log) - 1, h = hslot(x, log);
    for (uint32_t i = 0; i <= mask; i++) {
        uint32_t v = H[h];
        if (v == x + 1) return true;
        if (v == 0) return false;
        h = (h + 1) & mask;
    }
    return false;
}
// membership test that also reports where the probe ended: the slot holding
// x, or the empty slot an insertion of x would take (~0 if the table is full)
__device__ __forceinline__ bool hash_find(const uint32_t *H, uint32_t log, uint32_t x, uint32_t &slot) {
    uint32_t mask = (1u << log) - 1, h = hslot(x, log);
    for (uint32_t i = 0; i <= mask; i++) {
        uint32_t v = H[h];
        if (v == x + 1 || v == 0) {
            slot = h;
            return v != 0;
        }
        h = (h + 1) & mask;
    }
    slot = 0xffffffffu;
    return false;
}
__device__ __forceinline__ void hash_add(uint32_t *H, uint32_t log, uint32_t x) {
    uint32_t mask = (1u << log) - 1, h = hslot(x, log);
    for (uint32_t i = 0; i <= mask; i++) {
        uint32_t prev = atomicCAS(&H[h], 0u, x + 1);
        if (prev == 0 || prev == x + 1) return;
        h = (h + 1) & mask;
    }
}

// The same open-addressing table in global memory (large-budget kernels):
// one probe step reads the aligned 32-byte sector of eight slots holding the
// current slot, so an insertion or a lookup usually costs one memory round
// trip.  Only the owning warp reads and writes its table; plain loads and
// stores ordered by __syncwarp keep it coherent.  Returns as hash_find.
__device__ __forceinline__ bool ghash_find(const uint32_t *G, uint32_t log, uint32_t x, uint32_t &slot) {
    const uint32_t mask = (1u << log) - 1;
    uint32_t h = hslot(x, log), seen = 0;
    while (seen <= mask) {
        const uint32_t base = h & ~7u;
        const uint4 *p = (const uint4 *)(G + base);
        const uint4 a = __ldcg(p), b = __ldcg(p + 1);  // at L2: insertions by CAS bypass L1
        const uint32_t v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        uint32_t eq = 0, em = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            eq |= (uint32_t)(v[j] == x + 1) << j;
            em |= (uint32_t)(v[j] == 0) << j;
        }
        const uint32_t from = h & 7u;
        const uint32_t hit = ((eq | em) >> from) << from;
        if (hit) {
            const uint32_t j = __ffs(hit) - 1;
            slot = base + j;
            return (eq >> j) & 1u;
        }
        seen += 8 - from;
        h = (base + 8) & mask;
    }
    slot = 0xffffffffu;
    return false;
}
__device__ __forceinline__ bool ghash_has(const uint32_t *G, uint32_t log, uint32_t x) {
    uint32_t slot;
    return ghash_find(G, log, x, slot);
}

// ---------------------------------------------------------------------------
// main queue of reference entries (key << 32 | id): a 32-ary min-heap in
// shared memory.  Children of node i are 32i+1 .. 32i+32, so a pop reads one
// contiguous row of children per level and the warp finds their minimum with
// shuffles; a push appends and sifts up (rarely more than one level).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void warp_argmin(uint64_t &v, uint32_t &i) {
    // composite minimum with two warp reductions (key part, then id part)
    const uint32_t hi = (uint32_t)(v >> 32), lo = (uint32_t)v;
    const uint32_t mh = __reduce_min_sync(0xffffffffu, hi);
    const uint32_t ml = __reduce_min_sync(0xffffffffu, hi == mh ? lo : 0xffffffffu);
    const unsigned who = __ballot_sync(0xffffffffu, hi == mh && lo == ml);
    i = __shfl_sync(0xffffffffu, i, __ffs(who) - 1);
    v = ((uint64_t)mh << 32) | ml;
}

// remove the minimum (the caller has read h[0]); all lanes take part.  Per
// level: the smallest child key by one warp reduction; only when several
// children share it a second reduction over their ids.  The lane holding the
// smallest child moves it up.
__device__ __forceinline__ void heap_pop(uint64_t *h, uint32_t &sz) {
    const int lane = lane_id();
    sz--;
    const uint64_t v = h[sz];
    uint32_t i = 0;
    __syncwarp();
    for (;;) {
        const uint32_t c0 = 32 * i + 1;
        if (c0 >= sz) break;
        const uint32_t ci = c0 + lane;
        const uint64_t cv = ci < sz ? h[ci] : ~0ull;
        const uint32_t hi = (uint32_t)(cv >> 32);
        const uint32_t mh = __reduce_min_sync(0xffffffffu, hi);
        unsigned who = __ballot_sync(0xffffffffu, hi == mh);
        if (who & (who - 1)) {
            const uint32_t ml = __reduce_min_sync(0xffffffffu, hi == mh ? (uint32_t)cv : 0xffffffffu);
            who = __ballot_sync(0xffffffffu, hi == mh && (uint32_t)cv == ml);
        }
        const int w = __ffs(who) - 1;
        if (__ballot_sync(0xffffffffu, lane == w && cv >= v)) break;
        if (lane == w) h[i] = cv;
        i = c0 + (uint32_t)w;
    }
    __syncwarp();
    if (lane == 0 && sz > 0) h[i] = v;
    __syncwarp();
}

// append the entries of the lanes in `mask` (lane l holds entry e, stored at
// sz + pos, pos = its rank in the mask) and restore the heap order: every
// new entry checks its parent in parallel; those smaller than their parent
// sift up one after another (the new entries are leaves, or children of a
// new root, so any order of the sift-ups gives a valid heap)
__device__ __forceinline__ void heap_push_masked(uint64_t *h, uint32_t &sz, uint64_t e, unsigned mask, int pos) {
    const int lane = lane_id();
    const bool inm = (mask >> lane) & 1u;
    const uint32_t i0 = sz + (uint32_t)pos;
    if (inm) h[i0] = e;
    __syncwarp();
    const bool need = inm && i0 > 0 && h[(i0 - 1) >> 5] > e;
    unsigned nm = __ballot_sync(0xffffffffu, need);
    if (nm) {
        if (lane == 0) {
            while (nm) {
                const int j = __ffs(nm) - 1;
                nm &= nm - 1;
                uint32_t i = sz + __popc(mask & ((1u << j) - 1));
                const uint64_t val = h[i];
                while (i > 0) {
                    const uint32_t pi = (i - 1) >> 5;
                    const uint64_t pv = h[pi];
                    if (pv <= val) break;
                    h[i] = pv;
                    i = pi;
                }
                h[i] = val;
            }
        }
    }
    sz += __popc(mask);
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Spilling queue of the large-budget kernels.  The shared-memory heap holds
// the entries below a threshold tau; every entry >= tau sits, unsorted, in an
// overflow array in the warp's global scratch.  So whenever the heap is not
// empty its root is the minimum of the whole queue, and Algorithm 1's pop
// order is unchanged.  A full heap moves its upper part out (tau drops to a
// low quantile of 32 sampled entries); an empty heap takes the smallest
// overflow entries back (tau rises to a sampled quantile, checked by a count
// so that they fit).  Most discovered references are never popped, so the
// overflow is touched rarely.
// ---------------------------------------------------------------------------
struct Spill {
    uint64_t *B;   // overflow entries (global memory), unsorted, all >= tau
    uint32_t nb;   // their count (identical in every lane)
    uint64_t tau;  // heap entries < tau <= overflow entries; ~0 while nothing has spilled
};

// composite minimum of one 64-bit value per lane
__device__ __forceinline__ uint64_t warp_min64(uint64_t v) {
    const uint32_t hi = (uint32_t)(v >> 32), lo = (uint32_t)v;
    const uint32_t mh = __reduce_min_sync(0xffffffffu, hi);
    const uint32_t ml = __reduce_min_sync(0xffffffffu, hi == mh ? lo : 0xffffffffu);
    return ((uint64_t)mh << 32) | ml;
}

// restore the heap order below node i (all lanes take part)
__device__ inline void heap_sift_down(uint64_t *h, uint32_t sz, uint32_t i) {
    const int lane = lane_id();
    const uint64_t v = h[i];
    __syncwarp();
    for (;;) {
        const uint32_t c0 = 32 * i + 1;
        if (c0 >= sz) break;
        const uint32_t ci = c0 + lane;
        const uint64_t cv = ci < sz ? h[ci] : ~0ull;
        const uint64_t m = warp_min64(cv);
        const int w = __ffs(__ballot_sync(0xffffffffu, cv == m)) - 1;
        if (m >= v) break;
        if (lane == w) h[i] = cv;
        i = c0 + (uint32_t)w;
    }
    __syncwarp();
    if (lane == 0) h[i] = v;
    __syncwarp();
}

// bottom-up heap construction over h[0 .. sz)
__device__ inline void heap_build(uint64_t *h, uint32_t sz) {
    if (sz < 2) return;
    for (int64_t i = (int64_t)(sz - 2) / 32; i >= 0; i--) heap_sift_down(h, sz, (uint32_t)i);
}

// move the heap's entries >= t (a low sampled quantile) to the overflow
__device__ inline void spill_shrink(uint64_t *h, uint32_t &sz, Spill &sp) {
    const int lane = lane_id();
    const unsigned lt = (1u << lane) - 1;
    uint64_t smp[1] = {h[(uint32_t)(((uint64_t)lane * sz) >> 5)]};
    reg_bitonic_sort_t<1, uint64_t>(smp);
    const uint64_t t = __shfl_sync(0xffffffffu, smp[0], 12);  // an entry of the heap: at least it moves
    uint32_t w = 0, nb = sp.nb;
    for (uint32_t base = 0; base < sz; base += 32) {
        const uint32_t i = base + lane;
        const bool valid = i < sz;
        const uint64_t x = valid ? h[i] : ~0ull;
        const bool keep = valid && x < t;
        const unsigned mk = __ballot_sync(0xffffffffu, keep), mv = __ballot_sync(0xffffffffu, valid && !keep);
        __syncwarp();
        if (keep) h[w + __popc(mk & lt)] = x;  // in place: never past what this step read
        if (valid && !keep) sp.B[nb + __popc(mv & lt)] = x;
        w += __popc(mk);
        nb += __popc(mv);
        __syncwarp();
    }
    sz = w;
    sp.nb = nb;
    sp.tau = t;
    heap_build(h, sz);
}

// the heap is empty: take the smallest overflow entries back (at most hcap)
__device__ inline void spill_refill(uint64_t *h, uint32_t &sz, Spill &sp, uint32_t hcap) {
    const int lane = lane_id();
    const unsigned lt = (1u << lane) - 1;
    uint64_t t = ~0ull;  // everything fits: take it all
    if (sp.nb > hcap) {
        uint64_t smp[1] = {sp.B[(uint32_t)(((uint64_t)lane * sp.nb) >> 5)]};
        reg_bitonic_sort_t<1, uint64_t>(smp);
        int r = (int)((32u * (hcap / 2)) / sp.nb);  // the sample whose quantile is about hcap / 2 entries
        if (r > 31) r = 31;
        for (;;) {
            t = __shfl_sync(0xffffffffu, smp[0], r) + 1;  // entries up to that sample move
            uint32_t c = 0;
            for (uint32_t i = lane; i < sp.nb; i += 32) c += sp.B[i] < t;
            c = __reduce_add_sync(0xffffffffu, c);
            if (c <= hcap) break;
            if (r == 0) {
                uint64_t m = ~0ull;  // the exact minimum: one entry always fits
                for (uint32_t i = lane; i < sp.nb; i += 32) m = min(m, sp.B[i]);
                t = warp_min64(m) + 1;
                break;
            }
            r >>= 1;
        }
    }
    uint32_t na = 0, w = 0;
    for (uint32_t base = 0; base < sp.nb; base += 32) {
        const uint32_t i = base + lane;
        const bool valid = i < sp.nb;
        const uint64_t x = valid ? sp.B[i] : ~0ull;
        const bool in = valid && x < t;
        const unsigned mi = __ballot_sync(0xffffffffu, in), mo = __ballot_sync(0xffffffffu, valid && !in);
        __syncwarp();
        if (in) h[na + __popc(mi & lt)] = x;
        if (valid && !in) sp.B[w + __popc(mo & lt)] = x;  // compacted in place
        na += __popc(mi);
        w += __popc(mo);
        __syncwarp();
    }
    sz = na;
    sp.nb = w;
    sp.tau = w == 0 ? ~0ull : t;
    heap_build(h, sz);
}

template <bool SP>
__device__ __forceinline__ void queue_pop(uint64_t *h, uint32_t &sz, Spill &sp, uint32_t hcap) {
    heap_pop(h, sz);
    if (SP && sz == 0 && sp.nb > 0) spill_refill(h, sz, sp, hcap);
}

// push the entries of the lanes in mask (pos = the lane's rank in mask)
template <bool SP>
__device__ __forceinline__ void queue_push(uint64_t *h, uint32_t &sz, Spill &sp, uint32_t hcap, uint64_t e,
                                           unsigned mask, int pos) {
    if (!SP) {
        heap_push_masked(h, sz, e, mask, pos);
        return;
    }
    const int lane = lane_id();
    const unsigned lt = (1u << lane) - 1;
    const bool inm = (mask >> lane) & 1u;
    unsigned ma = __ballot_sync(0xffffffffu, inm && e < sp.tau);
    while (sz + __popc(ma) > hcap) {
        spill_shrink(h, sz, sp);
        ma = __ballot_sync(0xffffffffu, inm && e < sp.tau);
    }
    const unsigned mb = mask & ~ma;
    if (mb) {
        if ((mb >> lane) & 1u) sp.B[sp.nb + __popc(mb & lt)] = e;
        sp.nb += __popc(mb);
        __syncwarp();
    }
    if (ma) heap_push_masked(h, sz, e, ma, __popc(ma & lt));
    if (sz == 0 && sp.nb > 0) spill_refill(h, sz, sp, hcap);
}

// ---------------------------------------------------------------------------
// distances of candidate rows to the query.  cand[0..m) are row ids; keys go
// to ckey[0..m).  A group of G lanes (G = 16-byte chunks per row, at most 32)
// handles one row; all loads of several rows are issued before any is used.
// ---------------------------------------------------------------------------
template <int DT>
__device__ void cand_distances(const DevIndex &ix, const uint8_t *qbytes, const uint32_t *cand, int m,
                               uint32_t *ckey) {
    const int lane = lane_id();
    const int vb = ix.d * (DT == ANN_U8 ? 1 : 4);  // bytes per vector
    const int nc = vb >> 4;                          // 16-byte chunks
    int G = 1;
    while (G * 2 <= nc && G * 2 <= 32) G *= 2;
    const int per_round = 32 / G;
    const int lig = lane & (G - 1);
    const int grp = lane / G;
    const int cpl = (nc + G - 1) / G;                // chunks per lane per row
    constexpr int MAXL = 4;                          // 16-byte loads in flight per lane
    int rounds_per_batch = MAXL / cpl;
    if (rounds_per_batch < 1) rounds_per_batch = 1;
    const uint4 *qv = (const uint4 *)qbytes;
    if (cpl == 1 && G == nc) {
        // fast path: one 16-byte chunk per lane per row, MAXL rows' loads in flight
        const uint4 q = qv[lig];
        for (int base = 0; base < m; base += per_round * MAXL) {
            uint4 buf[MAXL];
#pragma unroll
            for (int u = 0; u < MAXL; u++) {
                const int j = base + u * per_round + grp;
                if (j < m) buf[u] = __ldg((const uint4 *)((const uint8_t *)ix.X + (int64_t)cand[j] * vb) + lig);
            }
#pragma unroll
            for (int u = 0; u < MAXL; u++) {
                const int j = base + u * per_round + grp;
                uint32_t acc = 0;
                float hi = 0.f, lo = 0.f;
                if (j < m) {
                    const uint4 a = buf[u];
                    if (DT == ANN_U8) {
                        uint32_t d0 = __vabsdiffu4(a.x, q.x), d1 = __vabsdiffu4(a.y, q.y);
                        uint32_t d2 = __vabsdiffu4(a.z, q.z), d3 = __vabsdiffu4(a.w, q.w);
                        acc = __dp4a(d0, d0, acc);
                        acc = __dp4a(d1, d1, acc);
                        acc = __dp4a(d2, d2, acc);
                        acc = __dp4a(d3, d3, acc);
                    } else {
                        df_acc_sqdiff(__uint_as_float(a.x), __uint_as_float(q.x), hi, lo);
                        df_acc_sqdiff(__uint_as_float(a.y), __uint_as_float(q.y), hi, lo);
                        df_acc_sqdiff(__uint_as_float(a.z), __uint_as_float(q.z), hi, lo);
                        df_acc_sqdiff(__uint_as_float(a.w), __uint_as_float(q.w), hi, lo);
                    }
                }
                for (int off = G >> 1; off > 0; off >>= 1) {
                    if (DT == ANN_U8) {
                        acc += __shfl_xor_sync(0xffffffffu, acc, off);
                    } else {
                        float h2 = __shfl_xor_sync(0xffffffffu, hi, off);
                        float l2 = __shfl_xor_sync(0xffffffffu, lo, off);
                        df_add(hi, lo, h2, l2);
                    }
                }
                if (j < m && lig == 0) ckey[j] = DT == ANN_U8 ? acc : __float_as_uint(__fadd_rn(hi, lo));
            }
            if (base + per_round * MAXL >= m) break;
        }
        __syncwarp();
        return;
    }
    for (int base = 0; base < m; base += per_round * rounds_per_batch) {
        uint4 buf[MAXL];
        // issue every load of this batch
#pragma unroll
        for (int u = 0; u < MAXL; u++) {
            int r = u / cpl, c = lig + (u % cpl) * G;
            int j = base + r * per_round + grp;
            if (r < rounds_per_batch && u < rounds_per_batch * cpl && j < m && c < nc)
                buf[u] = __ldg((const uint4 *)((const uint8_t *)ix.X + (int64_t)cand[j] * vb) + c);
        }
        // reduce row by row
        for (int r = 0; r < rounds_per_batch; r++) {
            int j = base + r * per_round + grp;
            uint32_t acc = 0;
            float hi = 0.f, lo = 0.f;
#pragma unroll
            for (int u = 0; u < MAXL; u++) {
                if (u / cpl != r || u >= rounds_per_batch * cpl) continue;
                int c = lig + (u % cpl) * G;
                if (j >= m || c >= nc) continue;
                uint4 a = buf[u], q = qv[c];
                if (DT == ANN_U8) {
                    uint32_t d0 = __vabsdiffu4(a.x, q.x), d1 = __vabsdiffu4(a.y, q.y);
                    uint32_t d2 = __vabsdiffu4(a.z, q.z), d3 = __vabsdiffu4(a.w, q.w);
                    acc = __dp4a(d0, d0, acc);
                    acc = __dp4a(d1, d1, acc);
                    acc = __dp4a(d2, d2, acc);
                    acc = __dp4a(d3, d3, acc);
                } else {
                    df_acc_sqdiff(__uint_as_float(a.x), __uint_as_float(q.x), hi, lo);
                    df_acc_sqdiff(__uint_as_float(a.y), __uint_as_float(q.y), hi, lo);
                    df_acc_sqdiff(__uint_as_float(a.z), __uint_as_float(q.z), hi, lo);
                    df_acc_sqdiff(__uint_as_float(a.w), __uint_as_float(q.w), hi, lo);
                }
            }
            // rows wider than MAXL chunks per lane: stream the rest
            if (cpl > MAXL && j < m) {
                const uint4 *row = (const uint4 *)((const uint8_t *)ix.X + (int64_t)cand[j] * vb);
                for (int c = lig + MAXL * G; c < nc; c += G) {
                    uint4 a = __ldg(row + c), q = qv[c];
                    if (DT == ANN_U8) {
                        uint32_t d0 = __vabsdiffu4(a.x, q.x), d1 = __vabsdiffu4(a.y, q.y);
                        uint32_t d2 = __vabsdiffu4(a.z, q.z), d3 = __vabsdiffu4(a.w, q.w);
                        acc = __dp4a(d0, d0, acc);
                        acc = __dp4a(d1, d1, acc);
                        acc = __dp4a(d2, d2, acc);
                        acc = __dp4a(d3, d3, acc);
                    } else {
                        df_acc_sqdiff(__uint_as_float(a.x), __uint_as_float(q.x), hi, lo);
                        df_acc_sqdiff(__uint_as_float(a.y), __uint_as_float(q.y), hi, lo);
                        df_acc_sqdiff(__uint_as_float(a.z), __uint_as_float(q.z), hi, lo);
                        df_acc_sqdiff(__uint_as_float(a.w), __uint_as_float(q.w), hi, lo);
                    }
                }
            }
            for (int off = G >> 1; off > 0; off >>= 1) {
                if (DT == ANN_U8) {
                    acc += __shfl_xor_sync(0xffffffffu, acc, off);
                } else {
                    float h2 = __shfl_xor_sync(0xffffffffu, hi, off);
                    float l2 = __shfl_xor_sync(0xffffffffu, lo, off);
                    df_add(hi, lo, h2, l2);
                }
            }
            if (j < m && lig == 0) ckey[j] = DT == ANN_U8 ? acc : __float_as_uint(__fadd_rn(hi, lo));
        }
    }
    __syncwarp();
}

// 16-byte asynchronous global -> shared copies (L2 only), completed per thread
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// squared distance of one row in shared memory to the query, by one lane
template <int DT>
__device__ __forceinline__ uint32_t row_key_smem(const uint8_t *row, const uint8_t *qbytes, int vb) {
    const uint4 *r = (const uint4 *)row, *qv = (const uint4 *)qbytes;
    const int nc = vb >> 4;
    if (DT == ANN_U8) {
        uint32_t a0 = 0, a1 = 0;
#pragma unroll 4
        for (int c = 0; c < nc; c++) {
            const uint4 a = r[c], q = qv[c];
            const uint32_t d0 = __vabsdiffu4(a.x, q.x), d1 = __vabsdiffu4(a.y, q.y);
            const uint32_t d2 = __vabsdiffu4(a.z, q.z), d3 = __vabsdiffu4(a.w, q.w);
            a0 = __dp4a(d0, d0, a0);
            a1 = __dp4a(d1, d1, a1);
            a0 = __dp4a(d2, d2, a0);
            a1 = __dp4a(d3, d3, a1);
        }
        return a0 + a1;
    } else {
        float hi = 0.f, lo = 0.f;
        for (int c = 0; c < nc; c++) {
            const uint4 a = r[c], q = qv[c];
            df_acc_sqdiff(__uint_as_float(a.x), __uint_as_float(q.x), hi, lo);
            df_acc_sqdiff(__uint_as_float(a.y), __uint_as_float(q.y), hi, lo);
            df_acc_sqdiff(__uint_as_float(a.z), __uint_as_float(q.z), hi, lo);
            df_acc_sqdiff(__uint_as_float(a.w), __uint_as_float(q.w), hi, lo);
        }
        return __float_as_uint(__fadd_rn(hi, lo));
    }
}

// ---------------------------------------------------------------------------
// bridge batch walk
// ---------------------------------------------------------------------------
struct WalkState {
    uint64_t lo;      // every non-empty bridge with composite <= lo has been produced
    bool first;       // nothing produced yet (lo meaningless)
    bool exhausted;   // all non-empty bridges produced
    uint32_t width;   // window width in key units (u8) or key-bit units (f32)
    uint32_t kmin, kmaxall, msuf;
    uint32_t gpos, gcnt;  // sorted window in global scratch: next entry, entries
    int gbuf;             // which of the two scratch buffers holds it
};

// A walk's output buffer is about to overflow: lower the window end hi to the
// median of 32 entries sampled from the buffer, keep the entries at or below
// it and let the walk go on with the lower end.  Entries are distinct
// (key, ranks) composites, so at least 16 leave the buffer, and the buffer
// ends up holding every bridge of (lo, final hi] -- no second walk needed.
__device__ inline void walk_trim(uint64_t *okey, uint32_t *oval, uint32_t *cnt, uint64_t &hi, uint32_t &hik) {
    const int lane = lane_id();
    const unsigned lt = (1u << lane) - 1;
    const uint32_t c = cnt[0];  // >= 32
    uint64_t smp[1] = {okey[(uint32_t)(((uint64_t)lane * c) >> 5)]};
    reg_bitonic_sort_t<1, uint64_t>(smp);
    const uint64_t t = __shfl_sync(0xffffffffu, smp[0], 15);
    uint32_t w = 0;
    for (uint32_t base = 0; base < c; base += 32) {
        const uint32_t i = base + lane;
        const bool valid = i < c;
        const uint64_t k = valid ? okey[i] : 0ull;
        const uint32_t v = valid ? oval[i] : 0u;
        const bool keep = valid && k <= t;
        const unsigned mk = __ballot_sync(0xffffffffu, keep);
        __syncwarp();
        if (keep) {  // in place: never past what this step read
            okey[w + __popc(mk & lt)] = k;
            oval[w + __popc(mk & lt)] = v;
        }
        w += __popc(mk);
        __syncwarp();
    }
    if (lane == 0) cnt[0] = w;
    hi = t;
    hik = (uint32_t)(t >> 32);
    __syncwarp();
}

// exclusive prefix sum over pref[0 .. n) in place, total in pref[n]
__device__ __forceinline__ void warp_exclusive_scan(uint32_t *pref, int n) {
    const int lane = lane_id();
    const int per = (n + 31) / 32;
    uint32_t local = 0;
    for (int i = 0; i < per; i++) {
        int r = lane * per + i;
        if (r < n) local += pref[r];
    }
    uint32_t incl = local;
    for (int off = 1; off < 32; off <<= 1) {
        uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    uint32_t run = incl - local;
    __syncwarp();
    for (int i = 0; i < per; i++) {
        int r = lane * per + i;
        if (r < n) {
            uint32_t v = pref[r];
            pref[r] = run;
            run += v;
        }
    }
    if (lane == 31) pref[n] = incl;
    __syncwarp();
}

// Second pass of a split walk (indexes with the suffix-major copy).  A bridge
// with prefix key A and suffix key B lies at or below hi only if A <= theta
// or B < hi - theta; the first pass read every bridge whose prefix bound is
// <= theta, so this pass lists the suffix nodes s with lower bound
// B(s) <= bound2 and keeps, of their bridges, only those whose prefix bound
// exceeds theta -- each bridge is read by exactly one pass that can emit it.
template <int DT>
__device__ void walk_suffix(const DevIndex &ix, uint8_t *smem, const WarpLayout &L, uint64_t lo, bool first,
                            uint64_t &hi, uint32_t theta, uint32_t bound2, uint64_t *okey, uint32_t *oval,
                            uint32_t ocap, int64_t &nodes_here, int64_t &leaves_here) {
    const int lane = lane_id();
    const int n = ix.n, P = ix.P, PA = ix.PA, q0 = ix.PA, nsuf = P - PA;
    const uint32_t *D = (const uint32_t *)(smem + L.tabD);
    const uint8_t *rk = smem + L.rank;
    const uint8_t *sc = smem + L.sc;
    auto sk = [&](int p, int r) -> uint32_t { return D[p * n + sc[p * n + r]]; };
    uint32_t *pref = (uint32_t *)(smem + L.pref);
    uint32_t *nodes = (uint32_t *)(smem + L.nodes);  // 4 words per node: start, count, key bound, (s << 16) | ranks
    uint32_t *cnt = (uint32_t *)(smem + L.misc);
    uint32_t hik = (uint32_t)(hi >> 32);
    const uint32_t lok = (uint32_t)(lo >> 32);
    const bool pow2n = (n & (n - 1)) == 0;
    const int logn = 31 - __clz(n);
    // candidate ranks of the second suffix part per rank of the first
    for (int r = lane; r < n; r += 32) {
        uint32_t c;
        if (nsuf == 1) {
            c = sk(q0, r) <= bound2 ? 1u : 0u;
        } else {
            const uint32_t b0 = sk(q0, r);
            if (KeyOps<DT>::add_lo(b0, sk(q0 + 1, 0)) > bound2) {
                c = 0;
            } else {
                int lo1 = 1, hi1 = n;
                while (lo1 < hi1) {
                    const int mid = (lo1 + hi1 + 1) >> 1;
                    if (KeyOps<DT>::add_lo(b0, sk(q0 + 1, mid - 1)) <= bound2) lo1 = mid;
                    else hi1 = mid - 1;
                }
                c = (uint32_t)lo1;
            }
        }
        pref[r] = c;
    }
    __syncwarp();
    warp_exclusive_scan(pref, n);
    const uint32_t total = pref[n];
    uint32_t nl = 0;
    int rp = 0;
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t f = base + lane;
        bool ok = false;
        uint32_t node = 0, kb = 0, rs = 0;
        if (f < total) {
            while (rp + 1 < n && pref[rp + 1] <= f) rp++;
            const int r2 = rp, r3 = (int)(f - pref[r2]);
            const uint32_t c2 = sc[q0 * n + r2];
            if (nsuf == 1) {
                node = c2;
                kb = D[q0 * n + c2];
                rs = (uint32_t)r2;
            } else {
                const uint32_t c3 = sc[(q0 + 1) * n + r3];
                node = c2 * n + c3;
                kb = KeyOps<DT>::add_lo(D[q0 * n + c2], D[(q0 + 1) * n + c3]);
                rs = ((uint32_t)r2 << 8) | (uint32_t)r3;
            }
            ok = (__ldg(ix.bmS + (node >> 5)) >> (node & 31)) & 1u;
        }
        nodes_here += (f < total);
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const uint32_t pos = nl + __popc(m & ((1u << lane) - 1));
            const uint32_t j0 = __ldg(ix.offS + node), j1 = __ldg(ix.offS + node + 1);
            nodes[4 * pos + 0] = j0;
            nodes[4 * pos + 1] = j1 - j0;
            nodes[4 * pos + 2] = kb;
            nodes[4 * pos + 3] = (node << 16) | rs;
        }
        nl += __popc(m);
        const bool flush = (nl + 32 > L.ncap) || (base + 32 >= total);
        if (!flush || nl == 0) continue;
        __syncwarp();
        uint32_t run = 0;
        for (uint32_t b0 = 0; b0 < nl; b0 += 32) {
            const uint32_t i = b0 + lane;
            const uint32_t c = i < nl ? nodes[4 * i + 1] : 0;
            uint32_t incl = c;
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += v;
            }
            if (i < nl) nodes[4 * i + 1] = run + incl - c;  // flat start of node i
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
        __syncwarp();
        uint32_t np = 0;
        constexpr int U2 = 2;  // leaf loads in flight per lane
        for (uint32_t b0 = 0; b0 < run; b0 += 32 * U2) {
            __syncwarp();
            while (cnt[0] + 32u * U2 > ocap) walk_trim(okey, oval, cnt, hi, hik);
            const uint32_t g0 = b0 + lane;
            uint32_t jjv[U2], av[U2], npv[U2];
#pragma unroll
            for (int u = 0; u < U2; u++) {
                const uint32_t g = g0 + 32 * u;
                jjv[u] = 0xffffffffu;
                if (g < run) {
                    while (np + 1 < nl && nodes[4 * (np + 1) + 1] <= g) np++;
                    npv[u] = np;
                    jjv[u] = nodes[4 * np + 0] + (g - nodes[4 * np + 1]);
                    av[u] = __ldg(ix.sleaf + jjv[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < U2; u++) {
                if (jjv[u] == 0xffffffffu) continue;
                const uint32_t jj = jjv[u], a = av[u], nq = npv[u];
                const uint32_t c0 = PA == 1 ? a : (pow2n ? (a >> logn) : a / n);
                const uint32_t c1 = PA == 1 ? 0u : a - c0 * n;
                const uint32_t kA = PA == 1 ? D[c0] : KeyOps<DT>::add_lo(D[c0], D[n + c1]);
                if (kA <= theta) continue;  // the first pass owns it
                const uint32_t kb = nodes[4 * nq + 2], sw = nodes[4 * nq + 3], sfx = sw >> 16;
                uint32_t key = KeyOps<DT>::add_lo(kA, kb);
                if (key > hik) continue;
                if (DT == ANN_F32) {
                    if (!first && KeyOps<DT>::add_hi(KeyOps<DT>::up(kA), KeyOps<DT>::up(kb)) < lok) continue;
                    uint32_t d1, d2 = 0u, d3 = 0u;
                    const uint32_t d0 = D[c0];
                    if (PA == 1) {
                        d1 = D[n + sfx];
                    } else {
                        d1 = D[n + c1];
                        if (nsuf == 1) {
                            d2 = D[2 * n + sfx];
                        } else {
                            const uint32_t c2 = pow2n ? (sfx >> logn) : sfx / n;
                            d2 = D[2 * n + c2];
                            d3 = D[3 * n + (sfx - c2 * n)];
                        }
                    }
                    key = KeyOps<DT>::sum4(d0, d1, d2, d3);
                    if (key > hik) continue;
                }
                if (!first && key < lok) continue;
                const uint32_t rpre = PA == 1 ? (uint32_t)rk[c0] : (((uint32_t)rk[c0] << 8) | rk[n + c1]);
                const uint32_t ranks = (rpre << (8 * nsuf)) | (sw & 0xffffu);
                const uint64_t comp = ((uint64_t)key << 32) | ranks;
                if (comp <= hi && (first || comp > lo)) {
                    const uint32_t slot = atomicAdd(&cnt[0], 1u);
                    if (slot < ocap) {
                        okey[slot] = comp;
                        oval[slot] = __ldg(ix.sidx + jj);
                    }
                }
            }
        }
        leaves_here += run;
        nl = 0;
        __syncwarp();
    }
}

// Emit the composite (key << 32 | packed ranks) of every non-empty bridge with
// lo < composite <= hi (lo ignored when first).  Returns how many there were;
// only the first ocap are stored.  Two phases per chunk: (1) the prefix
// nodes (c0[, c1]) whose lower bound fits the window and that hold bridges
// are collected into a node list; (2) the suffix leaves of the listed nodes
// are processed as one flat range, 32 consecutive leaves per step.  With the
// c2 group level (GRP), a phase between them keeps only the groups whose
// bound D0 + D1 + D2[c2] + min D3 fits the window, and (2) reads their leaves.
template <int DT, int UL, bool GRP>
__device__ uint32_t walk(const DevIndex &ix, uint8_t *smem, const WarpLayout &L, uint64_t lo, bool first,
                         uint64_t &hi, uint64_t *okey, uint32_t *oval,
                         uint32_t ocap) {
    const int lane = lane_id();
    const int n = ix.n, P = ix.P, PA = ix.PA;
    const uint32_t *D = (const uint32_t *)(smem + L.tabD);
    const uint8_t *rk = smem + L.rank;
    const uint8_t *sc = smem + L.sc;
    auto sk = [&](int i) -> uint32_t { return D[(i / n) * n + sc[i]]; };  // sorted key of prefix rank
    uint32_t *pref = (uint32_t *)(smem + L.pref);
    uint32_t *nodes = (uint32_t *)(smem + L.nodes);  // 4 words per node: start, count, kpre, rpre
    uint64_t *bkey = (uint64_t *)(smem + L.bkey);
    uint32_t *bidx = (uint32_t *)(smem + L.bidx);
    uint32_t *cnt = (uint32_t *)(smem + L.misc);
    uint32_t hik = (uint32_t)(hi >> 32);  // lowered, with hi, when the output buffer fills
    const bool pow2n = (n & (n - 1)) == 0;
    const int logn = 31 - __clz(n);
    const uint32_t msuf = cnt[3];     // min-suffix key sum, stored by the caller
    const uint32_t minlast = cnt[4];  // smallest key of the last part
    uint32_t *glist = (uint32_t *)(smem + L.glist);  // 5 words per group: start, count, kpre, D2, ranks
    const int nsuf = P - PA;
    if (lane == 0) cnt[0] = 0;
    // Split walk (suffix-major copy present, and a single pass would list
    // more than kSplitNodes prefix nodes): the first pass lists the prefix
    // nodes with bound A <= theta, the second (walk_suffix) the suffix nodes
    // with bound B <= bound2, so that A + B <= hi is covered by one of them;
    // theta splits the window's excess over the smallest possible A + B in
    // proportion to the parts on each side.  Otherwise one pass lists the
    // prefix nodes with A + min B <= hi (narrow windows: cheaper).
    constexpr uint32_t kSplitNodes = 256;
    const bool can_split = !GRP && ix.sidx != nullptr && L.sc_parts == (uint32_t)P;
    uint32_t theta = 0, bound2 = 0;
    bool pass2 = false;
    if (can_split) {
        const uint32_t minA = PA == 1 ? sk(0) : KeyOps<DT>::add_lo(sk(0), sk(n));
        if (DT == ANN_U8) {
            int64_t ex = (int64_t)hik - (int64_t)minA - (int64_t)msuf;
            if (ex < 0) ex = 0;
            int64_t th = (int64_t)minA + ex * PA / P;
            if (th > (int64_t)hik) th = hik;
            theta = (uint32_t)th;
            const int64_t b2 = (int64_t)hik - th - 1;  // integers: A > theta and A + B <= hi give B <= hi - theta - 1
            pass2 = b2 >= 0;
            bound2 = pass2 ? (uint32_t)b2 : 0u;
        } else {
            const float h = __uint_as_float(hik), a = __uint_as_float(minA), m = __uint_as_float(msuf);
            const float ex = fmaxf(h - a - m, 0.f);
            const float th = fminf(a + ex * (float)PA / (float)P, h);
            theta = __float_as_uint(th);
            // the key rounds the exact sum, so A + B < nextup(hi) when the key is <= hi
            const float b2 = __fsub_ru(__uint_as_float(f32_next_up(hik)), th);
            pass2 = b2 >= 0.f;
            bound2 = pass2 ? __float_as_uint(b2) : 0u;
        }
    }
    auto admit1 = [&](uint32_t kA) -> bool { return KeyOps<DT>::add_lo(kA, msuf) <= hik; };  // single pass
    auto admit2 = [&](uint32_t kA) -> bool { return kA <= theta; };                          // split
    // candidate part-1 ranks per r0 (PA == 2), or 0/1 per r0 (PA == 1), for
    // the single pass (pref) and the split (kept in the node area meanwhile)
    uint32_t *pref2 = nodes;
    uint32_t single_total = 0;
    for (int r0 = lane; r0 < n; r0 += 32) {
        uint32_t c1, c2 = 0;
        if (PA == 1) {
            c1 = admit1(sk(r0)) ? 1u : 0u;
            c2 = can_split && admit2(sk(r0)) ? 1u : 0u;
        } else {
            const uint32_t a0 = sk(r0);
            auto count = [&](bool two) -> uint32_t {
                if (!(two ? admit2(KeyOps<DT>::add_lo(a0, sk(n))) : admit1(KeyOps<DT>::add_lo(a0, sk(n))))) return 0;
                int lo1 = 1, hi1 = n;  // answer in [1, n]
                while (lo1 < hi1) {
                    const int mid = (lo1 + hi1 + 1) >> 1;
                    const uint32_t kA = KeyOps<DT>::add_lo(a0, sk(n + mid - 1));
                    if (two ? admit2(kA) : admit1(kA)) lo1 = mid;
                    else hi1 = mid - 1;
                }
                return (uint32_t)lo1;
            };
            c1 = count(false);
            if (can_split) c2 = count(true);
        }
        pref[r0] = c1;
        if (can_split) pref2[r0] = c2;  // the node area holds >= 256 words when the copy exists (no group level)
        single_total += c1;
    }
    single_total = __reduce_add_sync(0xffffffffu, single_total);
    const bool split = can_split && single_total > kSplitNodes;
    if (!split) pass2 = false;
    __syncwarp();
    if (split)
        for (int r0 = lane; r0 < n; r0 += 32) pref[r0] = pref2[r0];
    __syncwarp();
    warp_exclusive_scan(pref, n);
    const uint32_t total = pref[n];
    int64_t nodes_here = 0, leaves_here = 0;
    uint32_t nl = 0;      // listed nodes (warp-uniform)
    int r0p = 0;          // running r0 pointer of this lane
    for (uint32_t base = 0; base < total; base += 32) {
        uint32_t f = base + lane;
        bool ok = false;
        uint32_t node = 0, kpre = 0, rpre = 0;
        if (f < total) {
            while (r0p + 1 < n && pref[r0p + 1] <= f) r0p++;
            int r0 = r0p;
            int r1 = (int)(f - pref[r0]);
            uint32_t c0 = sc[r0];
            if (PA == 1) {
                node = c0;
                kpre = D[c0];
                rpre = (uint32_t)r0;
            } else {
                uint32_t c1 = sc[n + r1];
                node = c0 * n + c1;
                kpre = KeyOps<DT>::add_lo(D[c0], D[n + c1]);  // a lower bound for float32
                rpre = ((uint32_t)r0 << 8) | (uint32_t)r1;
            }
            ok = (__ldg(ix.bmA + (node >> 5)) >> (node & 31)) & 1u;
        }
        nodes_here += (f < total);
        unsigned m = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            uint32_t pos = nl + __popc(m & ((1u << lane) - 1));
            const uint32_t *off = GRP ? ix.goff : ix.offA;
            uint32_t j0 = __ldg(off + node), j1 = __ldg(off + node + 1);
            nodes[4 * pos + 0] = j0;
            nodes[4 * pos + 1] = j1 - j0;
            nodes[4 * pos + 2] = kpre;
            nodes[4 * pos + 3] = rpre;
        }
        nl += __popc(m);
        bool flush = (nl + 32 > L.ncap) || (base + 32 >= total);
        if (flush && nl > 0) {
            __syncwarp();
            // prefix over listed nodes' leaf counts (reuse the count word as its start in flat space)
            uint32_t run = 0;
            for (uint32_t b0 = 0; b0 < nl; b0 += 32) {
                uint32_t i = b0 + lane;
                uint32_t c = i < nl ? nodes[4 * i + 1] : 0;
                uint32_t incl = c;
                for (int off = 1; off < 32; off <<= 1) {
                    uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
                    if (lane >= off) incl += v;
                }
                if (i < nl) nodes[4 * i + 1] = run + incl - c;  // flat start of node i
                run += __shfl_sync(0xffffffffu, incl, 31);
            }
            __syncwarp();
            const uint32_t lt = run;
            uint32_t np = 0;  // running node pointer of this lane
            if (GRP) {
                // (1b) the c2 groups of the listed nodes (lt groups in flat space)
                uint32_t nlg = 0;  // listed groups (warp-uniform)
                for (uint32_t gb = 0; gb < lt; gb += 32) {
                    const uint32_t g = gb + lane;
                    bool okg = false;
                    uint32_t gi = 0, kp = 0, d2 = 0, rr = 0;
                    if (g < lt) {
                        while (np + 1 < nl && nodes[4 * (np + 1) + 1] <= g) np++;
                        gi = nodes[4 * np + 0] + (g - nodes[4 * np + 1]);
                        const uint32_t c2 = __ldg(ix.gc2 + gi);
                        kp = nodes[4 * np + 2];
                        d2 = D[2 * n + c2];
                        okg = KeyOps<DT>::add_lo(kp, KeyOps<DT>::add_lo(d2, minlast)) <= hik;
                        rr = (nodes[4 * np + 3] << 16) | ((uint32_t)rk[2 * n + c2] << 8);
                    }
                    const unsigned mg = __ballot_sync(0xffffffffu, okg);
                    if (okg) {
                        const uint32_t pos = nlg + __popc(mg & ((1u << lane) - 1));
                        const uint32_t s0 = __ldg(ix.gstart + gi), s1 = __ldg(ix.gstart + gi + 1);
                        glist[5 * pos + 0] = s0;
                        glist[5 * pos + 1] = s1 - s0;
                        glist[5 * pos + 2] = kp;
                        glist[5 * pos + 3] = d2;
                        glist[5 * pos + 4] = rr;
                    }
                    nlg += __popc(mg);
                    if ((nlg + 32 > L.gcap || gb + 32 >= lt) && nlg > 0) {
                        __syncwarp();
                        uint32_t grun = 0;
                        for (uint32_t b0 = 0; b0 < nlg; b0 += 32) {
                            const uint32_t i = b0 + lane;
                            const uint32_t c = i < nlg ? glist[5 * i + 1] : 0;
                            uint32_t incl = c;
                            for (int off = 1; off < 32; off <<= 1) {
                                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
                                if (lane >= off) incl += v;
                            }
                            if (i < nlg) glist[5 * i + 1] = grun + incl - c;  // flat start of group i
                            grun += __shfl_sync(0xffffffffu, incl, 31);
                        }
                        __syncwarp();
                        // (2) the leaves (c3) of the listed groups
                        uint32_t gp = 0;
                        for (uint32_t e0 = 0; e0 < grun; e0 += 32) {
                            __syncwarp();
                            while (cnt[0] + 32u > ocap) walk_trim(okey, oval, cnt, hi, hik);
                            const uint32_t e = e0 + lane;
                            if (e >= grun) continue;
                            while (gp + 1 < nlg && glist[5 * (gp + 1) + 1] <= e) gp++;
                            const uint32_t j = glist[5 * gp + 0] + (e - glist[5 * gp + 1]);
                            const uint32_t lf = __ldg(ix.leaf + j);
                            const uint32_t c3 = pow2n ? (lf & (uint32_t)(n - 1)) : lf % (uint32_t)n;
                            const uint32_t kp = glist[5 * gp + 2], d2 = glist[5 * gp + 3], d3 = D[3 * n + c3];
                            uint32_t key = KeyOps<DT>::add_lo(KeyOps<DT>::add_lo(kp, d2), d3);
                            if (key > hik) continue;
                            if (DT == ANN_F32) {
                                // bounds first; the exact key only for what may lie in the window
                                if (!first && KeyOps<DT>::add_hi(KeyOps<DT>::add_hi(KeyOps<DT>::up(kp), d2), d3) <
                                                  (uint32_t)(lo >> 32))
                                    continue;
                                const uint32_t rp = glist[5 * gp + 4] >> 16;
                                key = KeyOps<DT>::sum4(D[sc[rp >> 8]], D[n + sc[n + (rp & 255u)]], d2, d3);
                                if (key > hik) continue;
                            }
                            if (!first && key < (uint32_t)(lo >> 32)) continue;
                            const uint32_t ranks = glist[5 * gp + 4] | rk[3 * n + c3];
                            const uint64_t comp = ((uint64_t)key << 32) | ranks;
                            if (comp <= hi && (first || comp > lo)) {
                                const uint32_t s = atomicAdd(&cnt[0], 1u);
                                if (s < ocap) {
                                    okey[s] = comp;
                                    oval[s] = j;
                                }
                            }
                        }
                        leaves_here += grun;
                        nlg = 0;
                        __syncwarp();
                    }
                }
                nl = 0;
                __syncwarp();
                continue;
            }
            // UL leaves per lane per step, their loads in flight together
            for (uint32_t b0 = 0; b0 < lt; b0 += 32 * UL) {
                __syncwarp();
                while (cnt[0] + 32u * UL > ocap) walk_trim(okey, oval, cnt, hi, hik);
                const uint32_t g0 = b0 + lane;
                uint32_t jv[UL], lfv[UL], npv[UL];
#pragma unroll
                for (int u = 0; u < UL; u++) {
                    const uint32_t g = g0 + 32 * u;
                    jv[u] = 0xffffffffu;
                    if (g < lt) {
                        while (np + 1 < nl && nodes[4 * (np + 1) + 1] <= g) np++;
                        npv[u] = np;
                        jv[u] = nodes[4 * np + 0] + (g - nodes[4 * np + 1]);
                        lfv[u] = __ldg(ix.leaf + jv[u]);
                    }
                }
#pragma unroll
                for (int u = 0; u < UL; u++) {
                    if (jv[u] == 0xffffffffu) continue;
                    const uint32_t j = jv[u], lf = lfv[u], nq = npv[u];
                    // key first; the rank lookups only for keys inside the window
                    uint32_t c2 = 0, c3 = lf, ksuf;
                    if (nsuf == 1) {
                        ksuf = D[(P - 1) * n + lf];
                    } else {
                        c2 = pow2n ? (lf >> logn) : lf / n;
                        c3 = lf - c2 * n;
                        ksuf = KeyOps<DT>::add_lo(D[2 * n + c2], D[3 * n + c3]);
                    }
                    const uint32_t kpre = nodes[4 * nq + 2];
                    uint32_t key = KeyOps<DT>::add_lo(kpre, ksuf);
                    if (key > hik) continue;
                    if (DT == ANN_F32) {
                        // bounds first; the exact key only for what may lie in the window
                        if (!first && KeyOps<DT>::add_hi(KeyOps<DT>::up(kpre), KeyOps<DT>::up(ksuf)) <
                                          (uint32_t)(lo >> 32))
                            continue;
                        const uint32_t rp = nodes[4 * nq + 3];
                        const uint32_t d0 = PA == 1 ? D[sc[rp]] : D[sc[rp >> 8]];
                        const uint32_t d1 = PA == 1 ? D[n + lf] : D[n + sc[n + (rp & 255u)]];
                        const uint32_t d2 = PA == 1 ? 0u : (nsuf == 1 ? D[2 * n + lf] : D[2 * n + c2]);
                        const uint32_t d3 = nsuf == 2 ? D[3 * n + c3] : 0u;
                        key = KeyOps<DT>::sum4(d0, d1, d2, d3);
                        if (key > hik) continue;
                    }
                    if (!first && key < (uint32_t)(lo >> 32)) continue;
                    const uint32_t rsuf = nsuf == 1 ? (uint32_t)rk[(P - 1) * n + lf]
                                                    : (((uint32_t)rk[2 * n + c2] << 8) | rk[3 * n + c3]);
                    const uint32_t ranks = (nodes[4 * nq + 3] << (8 * nsuf)) | rsuf;
                    const uint64_t comp = ((uint64_t)key << 32) | ranks;
                    if (comp <= hi && (first || comp > lo)) {
                        const uint32_t s = atomicAdd(&cnt[0], 1u);
                        if (s < ocap) {
                            okey[s] = comp;
                            oval[s] = j;
                        }
                    }
                }
            }
            leaves_here += lt;
            nl = 0;
            __syncwarp();
        }
    }
    __syncwarp();
    if (!GRP && split && pass2)
        walk_suffix<DT>(ix, smem, L, lo, first, hi, theta, bound2, okey, oval, ocap, nodes_here, leaves_here);
    __syncwarp();
    for (int off = 16; off > 0; off >>= 1) nodes_here += __shfl_xor_sync(0xffffffffu, nodes_here, off);
    if (lane == 0) {
        cnt[8]++;
        cnt[9] += (uint32_t)nodes_here;
        cnt[10] += (uint32_t)leaves_here;
    }
    __syncwarp();
    return cnt[0];
}

// next window end (composite) from lo with width w, capped at the largest key
__device__ __forceinline__ uint64_t window_end(uint64_t lo, bool first, uint32_t kmin, uint32_t w,
                                               uint32_t kmaxall) {
    uint32_t base = first ? kmin : (uint32_t)(lo >> 32);
    uint64_t e = (uint64_t)base + (uint64_t)w;
    if (e > kmaxall) e = kmaxall;
    return (e << 32) | 0xffffffffull;
}

// The walk lowered the window end to fit its buffer: the next windows start
// at the width that window ended up with.
__device__ __forceinline__ void window_resize(WalkState &ws, uint64_t hi) {
    const uint32_t base = ws.first ? ws.kmin : (uint32_t)(ws.lo >> 32);
    const uint32_t w = (uint32_t)(hi >> 32) - base;
    ws.width = w > 1 ? w : 1;
}

// Refill the batch: bridges after ws.lo in order.  Returns count (0 = none left).
template <int DT, bool GRP>
__device__ uint32_t refill(const DevIndex &ix, uint8_t *smem, const WarpLayout &L, WalkState &ws,
                           bool &cap_err) {
    uint64_t *bkey = (uint64_t *)(smem + L.bkey);
    uint32_t *bidx = (uint32_t *)(smem + L.bidx);
    const int lane = lane_id();
    while (!ws.exhausted) {
        uint64_t hi = window_end(ws.lo, ws.first, ws.kmin, ws.width, ws.kmaxall);
        const uint64_t hi0 = hi;
        uint32_t c = walk<DT, 1, GRP>(ix, smem, L, ws.lo, ws.first, hi, bkey, bidx, L.bcap);
        if (hi != hi0) window_resize(ws, hi);
        if (c > L.bcap) {
            // too many in the window: halve it (in composite space).  A walk
            // lowers its own end before its buffer overflows, so this is a
            // guard only
            uint64_t base = ws.first ? ((uint64_t)ws.kmin << 32) : ws.lo + 1;
            uint64_t span = hi - base;
            if (span == 0) { cap_err = true; return 0; }
            // shrink the key width, or split inside one key by ranks
            if (ws.width > 1) {
                ws.width >>= 1;
                continue;
            }
            // width 1 key unit: split the composite range directly
            uint64_t h2 = base + span / 2;
            while (true) {
                c = walk<DT, 1, GRP>(ix, smem, L, ws.lo, ws.first, h2, bkey, bidx, L.bcap);
                        if (c <= L.bcap) break;
                span = h2 - base;
                if (span == 0) { cap_err = true; return 0; }
                h2 = base + span / 2;
            }
            hi = h2;
        }
        bool reached_end = (uint32_t)(hi >> 32) >= ws.kmaxall && (uint32_t)hi == 0xffffffffu;
        ws.lo = hi;
        ws.first = false;
        if (reached_end) ws.exhausted = true;
        if (c == 0) {
            if (ws.width < 0x40000000u) ws.width <<= 1;
            continue;
        }
        // grow the window while batches stay small
        if (c < L.bcap / 8 && ws.width < 0x40000000u) ws.width <<= 2;
        else if (c < L.bcap / 4 && ws.width < 0x40000000u) ws.width <<= 1;
        // sort the batch
        uint32_t Lp = 1;
        while (Lp < c) Lp <<= 1;
        for (uint32_t i = c + lane; i < Lp; i += 32) {
            bkey[i] = ~0ull;
            bidx[i] = 0;
        }
        __syncwarp();
        warp_sort_pairs(bkey, bidx, (int)Lp);
        return c;
    }
    return 0;
}

// Stable LSD radix sort of n (composite, index) pairs held in global scratch
// by one warp: 8-bit digits, passes whose digit is the same for every entry
// are skipped.  Returns the buffer (0 or 1) that holds the result.  cnt256:
// 256 shared-memory counters.
__device__ inline int warp_radix_sort(uint64_t *k0, uint32_t *v0, uint64_t *k1, uint32_t *v1, uint32_t n,
                               uint32_t *cnt256) {
    const int lane = lane_id();
    int cur = 0;
    for (int pass = 0; pass < 8; pass++) {
        const int sh = 8 * pass;
        uint64_t *ks = cur ? k1 : k0;
        uint32_t *vs = cur ? v1 : v0;
        uint64_t *kd = cur ? k0 : k1;
        uint32_t *vd = cur ? v0 : v1;
        for (int i = lane; i < 256; i += 32) cnt256[i] = 0;
        __syncwarp();
        for (uint32_t i = lane; i < n; i += 32) atomicAdd(&cnt256[(ks[i] >> sh) & 255], 1u);
        __syncwarp();
        // skip a pass whose digit is identical for all entries
        bool all_same = false;
        for (int i = lane; i < 256; i += 32) all_same |= cnt256[i] == n;
        if (__any_sync(0xffffffffu, all_same)) continue;
        // exclusive scan of the 256 counters (8 per lane)
        uint32_t loc[8], sum = 0;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            loc[i] = cnt256[lane * 8 + i];
            sum += loc[i];
        }
        uint32_t incl = sum;
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        uint32_t run = incl - sum;
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 8; i++) {
            cnt256[lane * 8 + i] = run;
            run += loc[i];
        }
        __syncwarp();
        // stable scatter, 32 entries at a time in input order
        for (uint32_t c0 = 0; c0 < n; c0 += 32) {
            const uint32_t i = c0 + lane;
            const bool valid = i < n;
            const uint64_t kv = valid ? ks[i] : 0;
            const uint32_t vv = valid ? vs[i] : 0;
            const uint32_t dig = valid ? (uint32_t)((kv >> sh) & 255) : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, dig);
            const int rank = __popc(peers & ((1u << lane) - 1));
            const uint32_t base = valid ? cnt256[dig] : 0;
            if (valid) {
                kd[base + rank] = kv;
                vd[base + rank] = vv;
            }
            __syncwarp();
            if (valid && rank == 0) cnt256[dig] = base + __popc(peers);
            __syncwarp();
        }
        cur ^= 1;
    }
    __syncwarp();
    return cur;
}

// Refill the shared-memory batch with the next bridges after ws.lo in order.
// A walk emits every non-empty bridge of a key window into the warp's global
// scratch (up to gcap), the window is sorted once, and the batch is served
// from it bcap entries at a time.  Returns the count (0 = none left).
template <int DT, bool GRP>
__device__ uint32_t refill_windowed(const DevIndex &ix, uint8_t *smem, const WarpLayout &L, WalkState &ws,
                                    bool &cap_err, uint8_t *wscratch, uint32_t gcap) {
    uint64_t *gk0 = (uint64_t *)wscratch;
    uint64_t *gk1 = gk0 + gcap;
    uint32_t *gv0 = (uint32_t *)(gk1 + gcap);
    uint32_t *gv1 = gv0 + gcap;
    uint64_t *bkey = (uint64_t *)(smem + L.bkey);
    uint32_t *bidx = (uint32_t *)(smem + L.bidx);
    const int lane = lane_id();
    if (ws.gpos >= ws.gcnt) {
        ws.gpos = ws.gcnt = 0;
        while (!ws.exhausted) {
            uint64_t hi = window_end(ws.lo, ws.first, ws.kmin, ws.width, ws.kmaxall);
            const uint64_t hi0 = hi;
            uint32_t c = walk<DT, 4, GRP>(ix, smem, L, ws.lo, ws.first, hi, gk0, gv0, gcap);
            if (hi != hi0) window_resize(ws, hi);
            if (c > gcap) {
                // too many in the window: halve it (in composite space).  A
                // walk lowers its own end before its buffer overflows, so this
                // is a guard only
                uint64_t base = ws.first ? ((uint64_t)ws.kmin << 32) : ws.lo + 1;
                uint64_t span = hi - base;
                if (span == 0) { cap_err = true; return 0; }
                if (ws.width > 1) {
                    ws.width >>= 1;
                    continue;
                }
                uint64_t h2 = base + span / 2;
                while (true) {
                    c = walk<DT, 4, GRP>(ix, smem, L, ws.lo, ws.first, h2, gk0, gv0, gcap);
                                if (c <= gcap) break;
                    span = h2 - base;
                    if (span == 0) { cap_err = true; return 0; }
                    h2 = base + span / 2;
                }
                hi = h2;
            }
            bool reached_end = (uint32_t)(hi >> 32) >= ws.kmaxall && (uint32_t)hi == 0xffffffffu;
            ws.lo = hi;
            ws.first = false;
            if (reached_end) ws.exhausted = true;
            if (c == 0) {
                if (ws.width < 0x40000000u) ws.width <<= 1;
                continue;
            }
            // grow the window while windows stay small
            if (c < gcap / 16 && ws.width < 0x40000000u) ws.width <<= 2;
            else if (c < gcap / 4 && ws.width < 0x40000000u) ws.width <<= 1;
            __syncwarp();
            ws.gbuf = c > L.bcap ? warp_radix_sort(gk0, gv0, gk1, gv1, c, (uint32_t *)(smem + L.nodes)) : 0;
            ws.gcnt = c;
            ws.gpos = 0;
            break;
        }
        if (ws.gcnt == 0) return 0;
    }
    // next batch: copy up to bcap entries of the sorted window into shared memory
    const uint64_t *gk = ws.gbuf ? gk1 : gk0;
    const uint32_t *gv = ws.gbuf ? gv1 : gv0;
    const uint32_t c = min(L.bcap, ws.gcnt - ws.gpos);
    for (uint32_t i = lane; i < c; i += 32) {
        bkey[i] = gk[ws.gpos + i];
        bidx[i] = gv[ws.gpos + i];
    }
    uint32_t Lp = 1;
    while (Lp < c) Lp <<= 1;
    for (uint32_t i = c + lane; i < Lp; i += 32) {
        bkey[i] = ~0ull;
        bidx[i] = 0;
    }
    __syncwarp();
    if (ws.gcnt <= L.bcap) warp_sort_pairs(bkey, bidx, (int)Lp);  // small window: sorted here
    ws.gpos += c;
    return c;
}

// Sort part p by (key, center id) in registers; write each center's rank and,
// for prefix parts, the center id at each rank; record the first/last key.
// PACK: uint8 part keys below 2^24 travel as one 32-bit word (key << 8 | id),
// which orders exactly like the (key, id) pair.
template <int EPL, bool PACK>
__device__ __forceinline__ void sort_part(const uint32_t *D, uint8_t *rk, uint8_t *sc, int p, int n, int PA,
                                          uint32_t *first_keys, uint32_t *last_keys) {
    // PA here: how many leading parts keep their centers in rank order
    const int lane = lane_id();
    using K = typename std::conditional<PACK, uint32_t, uint64_t>::type;
    constexpr int SH = PACK ? 8 : 32;
    K v[EPL];
#pragma unroll
    for (int s = 0; s < EPL; s++) {
        const int c = lane * EPL + s;
        v[s] = c < n ? (((K)D[p * n + c]) << SH) | (K)c : ~(K)0;
    }
    reg_bitonic_sort_t<EPL, K>(v);
#pragma unroll
    for (int s = 0; s < EPL; s++) {
        const int r = lane * EPL + s;
        if (r < n) {
            const uint32_t c = (uint32_t)(v[s] & (PACK ? 0xffu : 0xffffffffu));
            rk[p * n + c] = (uint8_t)r;
            if (p < PA) sc[p * n + r] = (uint8_t)c;
        }
    }
    first_keys[p] = (uint32_t)(__shfl_sync(0xffffffffu, v[0], 0) >> SH);
    K lastv = v[0];
#pragma unroll
    for (int s = 0; s < EPL; s++)
        if (s == (n - 1) % EPL) lastv = v[s];
    last_keys[p] = (uint32_t)(__shfl_sync(0xffffffffu, lastv, (n - 1) / EPL) >> SH);
}

template <int DT>
__device__ __forceinline__ void sort_parts(const uint32_t *D, uint8_t *rk, uint8_t *sc, int P, int n, int PA,
                                           int dp, uint32_t *first_keys, uint32_t *last_keys) {
    // uint8 part keys are at most dp * 255^2
    const bool pack = DT == ANN_U8 && (uint64_t)dp * 65025u < (1u << 24);
    for (int p = 0; p < P; p++) {
        if (pack) {
            if (n <= 32) sort_part<1, true>(D, rk, sc, p, n, PA, first_keys, last_keys);
            else if (n <= 64) sort_part<2, true>(D, rk, sc, p, n, PA, first_keys, last_keys);
            else if (n <= 128) sort_part<4, true>(D, rk, sc, p, n, PA, first_keys, last_keys);
            else sort_part<8, true>(D, rk, sc, p, n, PA, first_keys, last_keys);
        } else {
            if (n <= 32) sort_part<1, false>(D, rk, sc, p, n, PA, first_keys, last_keys);
            else if (n <= 64) sort_part<2, false>(D, rk, sc, p, n, PA, first_keys, last_keys);
            else if (n <= 128) sort_part<4, false>(D, rk, sc, p, n, PA, first_keys, last_keys);
            else sort_part<8, false>(D, rk, sc, p, n, PA, first_keys, last_keys);
        }
    }
}

// ---------------------------------------------------------------------------
// one query, one warp
// ---------------------------------------------------------------------------
template <int DT, bool WIN, bool GRP>
__device__ void search_one(const SearchArgs &A, uint8_t *smem, int64_t qi, uint8_t *wscratch) {
    constexpr bool SP = WIN;  // the large-budget kernels also spill the queue and the visited set
    const DevIndex &ix = A.ix;
    const WarpLayout &L = A.L;
    const int lane = lane_id();
    const int n = ix.n, P = ix.P, PA = ix.PA, dp = ix.d / ix.P;
    const int k = A.k ? A.k[qi] : A.k_all;
    const int T = A.T ? A.T[qi] : A.T_all;
    int32_t *oid = A.out_ids + qi * A.kmax;
    // per-query counters (registers; the walk keeps its own in shared memory)
    uint32_t n_refpops = 0, n_brpops = 0, n_ready = 0;
    if (k < 0 || k > A.kmax || T < 0 || T > A.capT) {
        for (int j = lane; j < A.kmax; j += 32) {
            oid[j] = -1;
            if (A.out_keys) ((uint32_t *)A.out_keys)[qi * A.kmax + j] = DT == ANN_U8 ? 0xffffffffu : 0x7f800000u;
        }
        if (A.out_status && lane == 0) A.out_status[qi] = ANN_ERR_ARG;
        return;
    }
    uint8_t *qb = smem + L.q;
    uint32_t *D = (uint32_t *)(smem + L.tabD);
    uint8_t *rk = smem + L.rank;
    uint8_t *sc = smem + L.sc;
    uint64_t *heap = (uint64_t *)(smem + L.heap);
    uint32_t *H = SP ? (uint32_t *)(wscratch + A.hash_off) : (uint32_t *)(smem + L.hash);
    Spill sp{SP ? (uint64_t *)(wscratch + A.spill_off) : nullptr, 0u, ~0ull};
    uint64_t *rbuf = (uint64_t *)(smem + L.rbuf);
    uint64_t *bkey = (uint64_t *)(smem + L.bkey);
    uint32_t *bidx = (uint32_t *)(smem + L.bidx);
    uint32_t *cand = (uint32_t *)(smem + L.cand);
    uint32_t *ckey = (uint32_t *)(smem + L.ckey);
    uint32_t *misc = (uint32_t *)(smem + L.misc);

    // load the query
    const int vb = ix.d * (DT == ANN_U8 ? 1 : 4);
    {
        const uint4 *src = (const uint4 *)((const uint8_t *)A.queries + qi * (int64_t)vb);
        uint4 *dst = (uint4 *)qb;
        for (int c = lane; c < (vb >> 4); c += 32) dst[c] = __ldg(src + c);
    }
    // clear the visited set and the walk counters
    if (SP) {
        for (uint32_t i = 4 * lane; i < (1u << L.hash_log); i += 128) *(uint4 *)(H + i) = make_uint4(0, 0, 0, 0);
    } else {
        for (uint32_t i = lane; i < (1u << L.hash_log); i += 32) H[i] = 0;
    }
    if (lane < 16) misc[lane] = 0;
    __syncwarp();

    // 1. part tables
    for (int idx = lane; idx < P * n; idx += 32) {
        int p = idx / n, c = idx % n;
        D[idx] = part_key_lane<DT>(qb, ix.C, p, c, n, dp);
    }
    __syncwarp();
    // 2. per-part sort by (key, center id); ranks for every part, sorted keys/ids for prefix parts
    uint32_t msuf = 0, minlast = 0;
    uint32_t kmin = 0, kmaxall = 0;
    {
        uint32_t first_keys[kMaxP], last_keys[kMaxP];
        sort_parts<DT>(D, rk, sc, P, n, (int)L.sc_parts, dp, first_keys, last_keys);
        __syncwarp();
        // smallest / largest bridge keys (exact sums) and a lower bound of the
        // smallest suffix sum
        auto key_sum = [&](const uint32_t *v) -> uint32_t {
            return KeyOps<DT>::sum4(v[0], v[1], P > 2 ? v[2] : 0u, P > 3 ? v[3] : 0u);
        };
        kmin = key_sum(first_keys);
        kmaxall = key_sum(last_keys);
        if (PA == 1) {
            msuf = first_keys[1];
        } else {
            msuf = first_keys[2];
            for (int p = 3; p < P; p++) msuf = KeyOps<DT>::add_lo(msuf, first_keys[p]);
        }
        minlast = first_keys[P - 1];
    }
    if (lane == 0) {
        misc[3] = msuf;
        misc[4] = minlast;
    }
    __syncwarp();

    // 3. Algorithm 1
    WalkState ws;
    ws.gpos = ws.gcnt = 0;
    ws.gbuf = 0;
    ws.lo = 0;
    ws.first = true;
    ws.exhausted = ix.M == 0;
    ws.kmin = kmin;
    ws.kmaxall = kmaxall;
    ws.msuf = msuf;
    if (DT == ANN_U8) {
        uint32_t w = kmin >> 8;  // measured on the SIFT-shaped 1M index: narrow first windows walk fewest leaves
        ws.width = w < 1 ? 1 : w;
    } else {
        ws.width = 1u << 16;  // about 0.8% relative in float32 bit space
    }
    uint32_t bcur = 0, bcnt = 0;
    uint32_t wstart = 0, wcnt = 0;  // bridge window: batch entries [wstart, wstart + wcnt)
    uint32_t wsize = 1;             // next window size: 1, 2, 4, ... 32 bridges
    uint32_t hsz = 0;               // heap size (identical in every lane)
    uint32_t rlen = 0;
    uint64_t rreg = ~0ull;          // result list in registers when k <= 32: lane l holds rank l
    const bool rsmall = k <= 32;
    int t = 0;
    bool cap_err = false;
    int64_t maxq = 0;
    const int b = ix.b, R = ix.R;
    int32_t *wref = (int32_t *)(smem + L.wref);
    uint32_t *wkey = (uint32_t *)(smem + L.wkey);
    // The next pop, once known, is staged: its kNN row in registers (nx_row)
    // and, when stage_rows > 0, its unvisited neighbours' vectors copied into
    // shared memory by cp.async (nx_vec, nx_mask = which row entries are new,
    // cut to the budget).  The vectors and mask stay valid only while nothing
    // else is discovered, i.e. for the very next step.  Right after every
    // reference pop the new heap root's row is loaded speculatively (sp_row):
    // it is the next pop unless the expansion finds a smaller key.
    constexpr uint32_t kNone = 0xffffffffu;
    uint32_t nx_id = kNone, sp_id = kNone;
    int32_t nx_row = -1, sp_row = -1;
    bool nx_vec = false, cp_out = false;
    unsigned nx_mask = 0;
    uint32_t nx_slot = kNone;  // where this lane's staged id goes in the visited set
    const int vbytes = ix.d * (DT == ANN_U8 ? 1 : 4);
    const int snc = vbytes >> 4;  // 16-byte chunks per row
    uint8_t *stage = smem + L.stage;

    while (t < T) {
        if (bcur >= bcnt && (!ws.exhausted || (WIN && ws.gpos < ws.gcnt))) {
            // the walk reuses the staging region
            if (cp_out) {
                cp_async_wait_all();
                cp_out = false;
            }
            nx_vec = false;
            __syncwarp();
            if (WIN) bcnt = refill_windowed<DT, GRP>(ix, smem, L, ws, cap_err, wscratch, A.gcap);
            else bcnt = refill<DT, GRP>(ix, smem, L, ws, cap_err);
            bcur = 0;
            wstart = 0;
            wcnt = 0;
            if (cap_err) break;
        }
        bool hb = bcur < bcnt;
        bool hr = hsz > 0;
        if (!hb && !hr) break;
        uint64_t top = hr ? heap[0] : ~0ull;
        uint64_t bc = hb ? bkey[bcur] : ~0ull;
        bool take_ref = hr && (!hb || (uint32_t)(top >> 32) <= (uint32_t)(bc >> 32));
        int32_t x = -1;
        uint32_t xkey = 0;
        bool have_key = false;
        bool staged = false;
        int alen;
        if (take_ref) {
            uint32_t p = (uint32_t)top;
            queue_pop<SP>(heap, hsz, sp, L.heap_cap);
            alen = R;
            if (p == nx_id) {
                x = nx_row;
                staged = nx_vec;
                n_ready++;
            } else if (p == sp_id) {
                x = sp_row;
                n_ready++;
            } else if (lane < R) {
                x = __ldg(ix.G + (int64_t)p * R + lane);
            }
            nx_id = kNone;
            nx_vec = false;
            if (hsz > 0) {
                sp_id = (uint32_t)heap[0];
                sp_row = lane < R ? __ldg(ix.G + (int64_t)sp_id * R + lane) : -1;
            } else {
                sp_id = kNone;
            }
            n_refpops++;
        } else {
            // the bridge window reuses the staging region
            if (cp_out) {
                cp_async_wait_all();
                cp_out = false;
            }
            nx_vec = false;
            __syncwarp();
            if (bcur >= wstart + wcnt) {
                // fill the window: reference lists of the next bridges and their distances
                wstart = bcur;
                wcnt = min(wsize, bcnt - bcur);
                if (wsize < 32) wsize <<= 1;
                for (int e = lane; e < (int)wcnt * b; e += 32) {
                    uint32_t j = bidx[wstart + e / b];
                    int32_t r = __ldg(ix.brefs + (int64_t)j * b + (e % b));
                    bool keep = r >= 0 && r < ix.N &&
                                !(SP ? ghash_has(H, L.hash_log, (uint32_t)r) : hash_has(H, L.hash_log, (uint32_t)r));
                    wref[e] = keep ? r : -1;
                }
                __syncwarp();
                int nc = 0;
                for (int e0 = 0; e0 < (int)wcnt * b; e0 += 32) {
                    int e = e0 + lane;
                    bool keep = e < (int)wcnt * b && wref[e] >= 0;
                    unsigned mk = __ballot_sync(0xffffffffu, keep);
                    if (keep) {
                        int pos = nc + __popc(mk & ((1u << lane) - 1));
                        cand[pos] = (uint32_t)wref[e];
                        wkey[e] = (uint32_t)pos;  // temporarily: where its key will land
                    }
                    nc += __popc(mk);
                }
                __syncwarp();
                cand_distances<DT>(ix, qb, cand, nc, ckey);
                for (int e = lane; e < (int)wcnt * b; e += 32)
                    if (wref[e] >= 0) wkey[e] = ckey[wkey[e]];
                __syncwarp();
            }
            uint32_t wi = (bcur - wstart) * b;
            bcur++;
            alen = b;
            if (lane < b) {
                x = wref[wi + lane];
                xkey = wkey[wi + lane];
            }
            have_key = true;
            n_brpops++;
        }
        // the new references of this adjacency list, in list order, cut to the budget
        unsigned mask;
        uint32_t slot = kNone;
        if (staged) {
            mask = nx_mask;  // computed one step earlier against the same visited set and budget
            slot = nx_slot;
        } else {
            bool isnew = false;
            if (lane < alen && x >= 0 && x < ix.N)
                isnew = !(SP ? ghash_find(H, L.hash_log, (uint32_t)x, slot) : hash_find(H, L.hash_log, (uint32_t)x, slot));
            mask = __ballot_sync(0xffffffffu, isnew);
            int room = T - t;
            while (__popc(mask) > room) mask &= ~(1u << (31 - __clz(mask)));  // keep the first `room` in list order
        }
        const int m = __popc(mask);
        const bool inm = (mask >> lane) & 1u;
        const int pos = __popc(mask & ((1u << lane) - 1));
        uint64_t mine = ~0ull;
        if (m > 0) {
            // mark them visited: the lowest lane among those whose probe ended on
            // the same empty slot stores there; the others insert by CAS after it
            const unsigned peers = __match_any_sync(0xffffffffu, inm ? slot : 0xfffffffeu);
            const bool direct = inm && slot != kNone && (peers & ((1u << lane) - 1)) == 0;
            if (direct) H[slot] = (uint32_t)x + 1;
            __syncwarp();
            if (inm && !direct) hash_add(H, L.hash_log, (uint32_t)x);
            uint32_t key = xkey;
            if (!have_key) {
                if (staged) {
                    cp_async_wait_all();
                    cp_out = false;
                    __syncwarp();
                    if (inm) key = row_key_smem<DT>(stage + (size_t)pos * L.stage_stride, qb, vbytes);
                } else {
                    if (inm) cand[pos] = (uint32_t)x;
                    __syncwarp();
                    cand_distances<DT>(ix, qb, cand, m, ckey);
                    if (inm) key = ckey[pos];
                }
            }
            mine = inm ? (((uint64_t)key << 32) | (uint32_t)x) : ~0ull;
            queue_push<SP>(heap, hsz, sp, L.heap_cap, mine, mask, pos);
            if ((int64_t)hsz + sp.nb + 1 > maxq) maxq = (int64_t)hsz + sp.nb + 1;
        }
        // The next pop is known now.  When it is a reference, take its kNN row
        // (usually the speculative one) and start copying its unvisited
        // neighbours' vectors, so both overlap the rest of this step and the
        // next pop.
        if (t + m < T && hsz > 0) {
            const uint64_t ntop = heap[0];
            const bool maybe_ref = bcur >= bcnt || (uint32_t)(ntop >> 32) <= (uint32_t)(bkey[bcur] >> 32);
            if (maybe_ref) {
                const uint32_t nid = (uint32_t)ntop;
                if (nid != nx_id) {
                    nx_row = nid == sp_id ? sp_row : (lane < R ? __ldg(ix.G + (int64_t)nid * R + lane) : -1);
                    nx_id = nid;
                }
                // vectors only when the next step is certainly this pop (no
                // refill first) and no bridge-window entries are still pending
                const bool refill_next = bcur >= bcnt && (!ws.exhausted || (WIN && ws.gpos < ws.gcnt));
                if (L.stage_rows && !refill_next && bcur >= wstart + wcnt) {
                    uint32_t s2 = kNone;
                    bool nw = false;
                    if (lane < R && nx_row >= 0 && nx_row < ix.N)
                        nw = !(SP ? ghash_find(H, L.hash_log, (uint32_t)nx_row, s2)
                                  : hash_find(H, L.hash_log, (uint32_t)nx_row, s2));
                    unsigned mk = __ballot_sync(0xffffffffu, nw);
                    const int room2 = T - (t + m);
                    while (__popc(mk) > room2) mk &= ~(1u << (31 - __clz(mk)));
                    nx_mask = mk;
                    nx_slot = s2;
                    nx_vec = true;
                    if ((mk >> lane) & 1u) {
                        // each lane copies its own row into its rank's slot
                        const uint8_t *src = (const uint8_t *)ix.X + (int64_t)nx_row * vbytes;
                        uint8_t *dst = stage + (size_t)__popc(mk & ((1u << lane) - 1)) * L.stage_stride;
                        for (int c = 0; c < snc; c++) cp_async16(dst + 16 * c, src + 16 * c);
                    }
                    cp_async_commit();
                    cp_out = mk != 0;
                }
            }
        }
        if (m == 0) continue;
        // result set: the k smallest by (key, id)
        if (rsmall) {
            if (k > 0) {
                uint64_t kth = __shfl_sync(0xffffffffu, rreg, k - 1);  // ~0 while fewer than k
                unsigned pm = __ballot_sync(0xffffffffu, inm && mine < kth);
                while (pm) {
                    int j = __ffs(pm) - 1;
                    pm &= pm - 1;
                    uint64_t e = __shfl_sync(0xffffffffu, mine, j);
                    kth = __shfl_sync(0xffffffffu, rreg, k - 1);
                    if (e >= kth) continue;
                    int pos = __popc(__ballot_sync(0xffffffffu, rreg < e));
                    uint64_t up = __shfl_up_sync(0xffffffffu, rreg, 1);
                    if (lane == pos) rreg = e;
                    else if (lane > pos) rreg = up;
                    if ((int)rlen < k) rlen++;
                }
            }
        } else {
            for (unsigned pm = mask; pm; pm &= pm - 1) {
                const uint64_t e = __shfl_sync(0xffffffffu, mine, __ffs(pm) - 1);
                if ((int)rlen == k && e >= rbuf[k - 1]) continue;
                // position = number of entries smaller than e
                int cntless = 0;
                for (int i = lane; i < (int)rlen; i += 32) cntless += rbuf[i] < e;
                for (int off = 16; off > 0; off >>= 1) cntless += __shfl_xor_sync(0xffffffffu, cntless, off);
                int newlen = (int)rlen < k ? (int)rlen + 1 : k;
                // shift [cntless, newlen-1) up by one, top-down in chunks of 32
                for (int top_i = newlen - 1; top_i > cntless; top_i -= 32) {
                    int i = top_i - lane;
                    uint64_t v = 0;
                    bool mv = i > cntless;
                    if (mv) v = rbuf[i - 1];
                    __syncwarp();
                    if (mv) rbuf[i] = v;
                    __syncwarp();
                }
                if (lane == 0) rbuf[cntless] = e;
                rlen = (uint32_t)newlen;
                __syncwarp();
            }
        }
        t += m;
    }
    // nothing may still land in shared memory once this query ends
    if (cp_out) cp_async_wait_all();
    __syncwarp();
    if (rsmall) {
        if (lane < k) rbuf[lane] = rreg;
        __syncwarp();
    }
    __syncwarp();
    // outputs
    for (int j = lane; j < A.kmax; j += 32) {
        bool have = j < (int)rlen && j < k;
        oid[j] = have ? (int32_t)(uint32_t)rbuf[j] : -1;
        if (A.out_keys) {
            uint32_t kv = have ? (uint32_t)(rbuf[j] >> 32) : (DT == ANN_U8 ? 0xffffffffu : 0x7f800000u);
            ((uint32_t *)A.out_keys)[qi * A.kmax + j] = kv;
        }
    }
    if (lane == 0) {
        if (A.out_status) A.out_status[qi] = cap_err ? ANN_ERR_CAPACITY : ANN_OK;
        if (A.out_stats) {
            int64_t *o = A.out_stats + qi * ANN_NSTATS;
            o[ANN_STAT_DISCOVERED] = t;
            o[ANN_STAT_REF_POPS] = n_refpops;
            o[ANN_STAT_BRIDGE_POPS] = n_brpops;
            o[ANN_STAT_WALKS] = misc[8];
            o[ANN_STAT_WALK_NODES] = misc[9];
            o[ANN_STAT_WALK_LEAVES] = misc[10];
            o[ANN_STAT_MAX_Q] = maxq;
            o[ANN_STAT_PRELOADED] = n_ready;
        }
    }
    __syncwarp();
}

template <int DT, bool WIN, bool GRP>
__global__ void __launch_bounds__(192, 2) search_kernel(SearchArgs A) {
    extern __shared__ __align__(16) uint8_t smem_all[];
    const int warp = threadIdx.x >> 5;
    uint8_t *smem = smem_all + (size_t)warp * A.L.total;
    uint8_t *wscratch = WIN ? A.gscratch + ((size_t)blockIdx.x * (blockDim.x >> 5) + warp) * A.wstride : nullptr;
    const int64_t count = A.list_count ? (int64_t)*A.list_count : (A.list ? A.list_len : A.nq);
    if (A.ticket) {
        // persistent: pull queries from the device work queue
        for (;;) {
            int32_t w = 0;
            if (lane_id() == 0) w = atomicAdd(A.ticket, 1);
            w = __shfl_sync(0xffffffffu, w, 0);
            if (w >= count) break;
            int64_t qi = A.list ? A.list[w] : w;
            search_one<DT, WIN, GRP>(A, smem, qi, wscratch);
        }
    } else {
        const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
        const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
        for (int64_t w = gw; w < count; w += nw) {
            int64_t qi = A.list ? A.list[w] : w;
            search_one<DT, WIN, GRP>(A, smem, qi, wscratch);
        }
    }
}

// Launch helpers of the kernels with the c2 group level (ann_search_grp.cu).
cudaError_t config_grouped(int dtype, bool win, size_t smem, int threads, int *blocks_per_sm);
void launch_grouped(int dtype, bool win, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const SearchArgs &A);

}  // namespace ann
