// Middle-vertex shared-memory hash variant of the block-tuple kernel
// (PGAbB Section 3.6, which allows the intersection to be done over sorted
// lists or through a hash map).
//
// The TC device kernel (Section 3.6, Listing 5) loops over u, then over v in N(u), intersecting u's and
// v's partial lists.  This variant interchanges the two outer loops: a CTA
// takes a middle vertex v (or a group of up to 32 consecutive middle
// vertices), puts v's partial list N+(v) ∩ [lo, hi) into a shared-memory
// hash table once, then streams every in-neighbour u's list after v and
// looks each element up in the table.  A triangle u < v < w is found once,
// as the element w of u's list that hits v's table.  Each lookup costs one
// or two shared-memory loads instead of a chain of dependent global loads,
// and u's list is read with coalesced loads.
//
// Work items (built on the device, heaviest middle vertices first):
//   group item:     up to 32 consecutive ranks whose partial lists hold at
//                   most K entries in total (K: the table capacity of the
//                   CTA shape) and whose in-edges number at most in_chunk;
//                   table entries carry a 32-bit mask of the group members
//                   that own the key;
//   singleton item: one middle vertex, a run of at most in_chunk of its
//                   in-edges, and a slice of at most K entries of its
//                   list (the slice is a third-vertex rank range [lo, hi),
//                   i.e. a narrower column-block run; both lists are clipped).
// Per-vertex counts: a shared counter per table slot collects t[w], a
// per-edge tally collects t[u] and t[v]; all are flushed with one global
// atomic per (slot, item) and per in-edge instead of one per triangle.
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <type_traits>

#include "internal.cuh"
#include "tc_hash.cuh"

namespace pgb {

namespace {

constexpr uint32_t kInChunkDefault = 4096;  // in-edges per item unless the caller sets one
// At most this many in-edges per item: a key's per-vertex counter counts at
// most one hit per in-edge of the item and is 16 bits wide.
constexpr uint32_t kInChunkMax = 65535;
constexpr uint32_t kEmpty = 0xffffffffu;
constexpr int kModeDense = 0, kModeBitmap = 1, kModeTable = 2;  // an item's lookup structure
constexpr unsigned kFullMask = 0xffffffffu;
// Table keys per work item of a CTA shape (tables stay at most half full),
// and its bitmap bits (a third-vertex range narrower than that is held as a
// bitmap).
constexpr uint32_t key_capacity(int threads) { return 32u * threads / 4; }
constexpr uint32_t bitmap_range(int threads) { return 32u * 32u * threads; }

// Graphs with at least this many vertices run the 256-thread shape, and
// with at least kWidestShapeVertices the 512-thread one: their wider bitmaps
// and larger tables serve more of the top-ranked middle vertices (measured on
// R-MAT kernels: 256 threads is 10% faster than 128 at scale 24, 128 is 9%
// faster at scale 23; 512 is 11% faster than 256 at scale 26 and 23% at 27,
// 256 is 9% faster at scale 25 and 33% at 24).
constexpr uint32_t kWideShapeVertices = 1u << 24;
constexpr uint32_t kWidestShapeVertices = 1u << 26;
constexpr int kPairSlots = 3;          // 32-byte loads (8 entries) per lane issued together

__device__ __forceinline__ uint32_t hslot(uint32_t x, uint32_t log2s) { return (x * 0x9E3779B1u) >> (32 - log2s); }

__device__ __forceinline__ uint32_t ceil_log2(uint32_t x) { return x <= 1 ? 0 : 32 - __clz(x - 1); }

// Table slots (log2) of an item with `keys` keys: at most a quarter full
// where the capacity (2 * keycap slots) allows, else at most half full.
__device__ __forceinline__ uint32_t slots_for(uint32_t keys, uint32_t keycap) {
    uint32_t l = min(ceil_log2(4 * keys), ceil_log2(2 * keycap));
    return l < 6 ? 6 : l;
}

__device__ __forceinline__ uint32_t hlower_bound(const uint32_t* __restrict__ a, uint32_t b, uint32_t e, uint32_t x) {
    uint32_t n = e - b;
    while (n > 0) {
        uint32_t half = n >> 1;
        if (__ldg(a + b + half) < x) {
            b += half + 1;
            n -= half + 1;
        } else {
            n = half;
        }
    }
    return b;
}

// hlower_bound over an array whose entry q is stored at a[q - base].
__device__ __forceinline__ uint32_t hlower_bound_b(const uint32_t* __restrict__ a, uint32_t base, uint32_t b,
                                                   uint32_t e, uint32_t x) {
    return hlower_bound(a, b - base, e - base, x) + base;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFullMask, x, o);
    return x;
}

// Insert x into the open-addressing table (linear probing) and set `bit` in
// its member mask.  The table is never more than half full, so a free slot
// is always found.
__device__ __forceinline__ void table_insert(uint32_t* keys, uint32_t* masks, uint32_t x, uint32_t bit, uint32_t L) {
    const uint32_t smask = (1u << L) - 1;
    uint32_t h = hslot(x, L);
    for (uint32_t probe = 0; probe <= smask; ++probe) {
        const uint32_t old = atomicCAS(&keys[h], kEmpty, x);
        if (old == kEmpty || old == x) {
            if (bit) atomicOr(&masks[h], bit);
            return;
        }
        h = (h + 1) & smask;
    }
}

// Slot of x in the table, or kEmpty when x is absent.
__device__ __forceinline__ uint32_t table_find(const uint32_t* keys, uint32_t x, uint32_t L) {
    const uint32_t smask = (1u << L) - 1;
    uint32_t h = hslot(x, L);
    for (uint32_t probe = 0; probe <= smask; ++probe) {
        const uint32_t k = keys[h];
        if (k == x) return h;
        if (k == kEmpty) return kEmpty;
        h = (h + 1) & smask;
    }
    return kEmpty;
}

// Item decisions for the window of 32 ranks starting at w0 + 32 w (one warp).
// A window whose active lists fit one table is one group item.  Otherwise:
//   - a lane too big for one item (more keys than the capacity or more
//     in-edges than in_chunk), or whose range fits a bitmap, is a singleton,
//     split into in-edge chunks and key slices;
//   - the other active lanes ("light") form runs of consecutive ranks whose
//     keys fit one table and whose in-edges fit in_chunk, scanned greedily in
//     rank order; a run of two or more is a group item, a run of one a
//     singleton.  Without runs, mid-rank windows would give one small item
//     per vertex, each paying the per-item barriers.
struct WindowInfo {
    uint32_t v, dp, dm;
    bool act;
    uint32_t keys, ins;  // the whole window's active lanes
    bool group;          // the whole window is one group item
    uint32_t mine;       // items this lane emits
    uint32_t run_len, run_mask, run_keys;  // a run starting at this lane (run_len > 0)
};

// Whether head v is counted by this kernel under the per-part filter.
__device__ __forceinline__ bool head_selected(const ItemSpace& sp, uint32_t v) {
    if (!sp.part_hash) return true;
    uint32_t lo = 0, hi = sp.p;  // largest j in [0, p) with cuts[j] <= v
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(sp.cuts + mid) <= v) lo = mid; else hi = mid;
    }
    return __ldg(sp.part_hash + lo) != 0;
}

__device__ __forceinline__ WindowInfo window_info(const ItemSpace& sp, uint32_t w, uint32_t in_chunk, int lane) {
    WindowInfo W;
    W.v = sp.w0 + w * 32 + lane;
    W.dp = W.dm = 0;
    if (W.v < sp.n) {
        // a head outside the filter keeps its in-edges (they lie inside any
        // run's range) but no list, so it is never an active member
        W.dp = head_selected(sp, W.v) ? sp.rowptr[W.v + 1] - sp.rowptr[W.v] : 0;
        W.dm = sp.colptr[W.v + 1 - sp.cbase] - sp.colptr[W.v - sp.cbase];
    }
    W.act = W.dp > 0 && W.dm > 0;
    W.keys = warp_sum(W.act ? W.dp : 0);
    W.ins = warp_sum(W.act ? W.dm : 0);
    W.group = W.keys > 0 && W.keys <= sp.keycap && W.ins <= in_chunk;
    W.run_len = W.run_mask = W.run_keys = 0;
    W.mine = 0;
    if (W.group || W.keys == 0) return W;
    const bool light = W.act && W.dp <= sp.keycap && W.dm <= in_chunk && sp.n - W.v - 1 >= sp.bitmap_bits;
    const bool heavy = W.act && !light;
    if (heavy) W.mine = ((W.dm + in_chunk - 1) / in_chunk) * ((W.dp + sp.keycap - 1) / sp.keycap);
    // the same greedy scan in every lane (uniform), each keeping its own run
    uint32_t rs = 32, rlast = 0, rk = 0, ri = 0, rm = 0;
    auto close = [&] {
        if (rs < 32 && lane == (int)rs) {
            W.run_len = rlast - rs + 1;
            W.run_mask = rm;
            W.run_keys = rk;
            W.mine = 1;
        }
        rs = 32;
    };
    for (uint32_t t = 0; t < 32; ++t) {
        const bool lt = __shfl_sync(kFullMask, light, t);
        const bool ht = __shfl_sync(kFullMask, heavy, t);
        const uint32_t dpt = __shfl_sync(kFullMask, W.dp, t);
        const uint32_t dmt = __shfl_sync(kFullMask, W.dm, t);
        if (ht) {
            close();
        } else if (lt) {
            if (rs < 32 && (rk + dpt > sp.keycap || ri + dmt > in_chunk)) close();
            if (rs == 32) {
                rs = t;
                rk = ri = rm = 0;
            }
            rk += dpt;
            ri += dmt;
            rm |= 1u << (t - rs);
            rlast = t;
        } else if (rs < 32) {
            // an inactive lane inside a run: its in-edges lie in the run's range
            if (ri + dmt > in_chunk) close();
            else ri += dmt;
        }
    }
    close();
    return W;
}

// counts[nwin - 1 - w] = items of window w (windows of high ranks first).
__global__ void k_items_count(const ItemSpace sp, uint32_t in_chunk, uint32_t* __restrict__ counts) {
    const int lane = threadIdx.x & 31;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < sp.nwin; w += nw) {
        WindowInfo W = window_info(sp, w, in_chunk, lane);
        uint32_t c = W.keys == 0 ? 0 : (W.group ? 1 : warp_sum(W.mine));
        if (lane == 0) counts[sp.nwin - 1 - w] = c;
    }
}

__device__ __forceinline__ VItem group_item(const ItemSpace& sp, uint32_t v0, uint32_t nv, uint32_t keys,
                                            uint32_t mask) {
    VItem it;
    it.v0 = v0;
    it.nv = nv;
    it.in_begin = sp.colptr[v0 - sp.cbase];
    it.in_end = sp.colptr[v0 + nv - sp.cbase];
    it.lo = 0;
    it.hi = sp.n;
    it.slots_log2 = (uint16_t)slots_for(keys, sp.keycap);
    it.clip = 0;
    it.mask = mask;
    return it;
}

__global__ void k_items_emit(const ItemSpace sp, uint32_t in_chunk, const uint32_t* __restrict__ offs,
                             VItem* __restrict__ items) {
    const int lane = threadIdx.x & 31;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t n = sp.n;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < sp.nwin; w += nw) {
        WindowInfo W = window_info(sp, w, in_chunk, lane);
        if (W.keys == 0) continue;
        const uint32_t base = offs[sp.nwin - 1 - w];
        const unsigned act = __ballot_sync(kFullMask, W.act);
        if (W.group) {
            if (lane == 0) {
                const uint32_t v0 = sp.w0 + w * 32;
                items[base] = group_item(sp, v0, min(32u, n - v0), W.keys, act);
            }
            continue;
        }
        uint32_t excl = W.mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFullMask, excl, o);
            if (lane >= o) excl += y;
        }
        excl -= W.mine;
        if (!W.mine) continue;
        uint32_t out = base + excl;
        if (W.run_len > 1) {
            items[out] = group_item(sp, W.v, W.run_len, W.run_keys, W.run_mask);
            continue;
        }
        // a singleton: in-edge chunks times key slices
        const uint32_t na = (W.dm + in_chunk - 1) / in_chunk;
        const uint32_t kc = sp.keycap;
        const uint32_t nk = (W.dp + kc - 1) / kc;
        const uint32_t rb = sp.rowptr[W.v], cb = sp.colptr[W.v - sp.cbase];
        for (uint32_t a = 0; a < na; ++a) {
            for (uint32_t kk = 0; kk < nk; ++kk) {
                VItem it;
                it.v0 = W.v;
                it.nv = 1;
                it.in_begin = cb + a * in_chunk;
                it.in_end = min(it.in_begin + in_chunk, cb + W.dm);
                if (nk > 1) {
                    it.lo = sp.col[rb + kk * kc - sp.vbase];
                    it.hi = (kk + 1 < nk) ? sp.col[rb + (kk + 1) * kc - sp.vbase] : n;
                    it.clip = 1;
                } else {
                    it.lo = 0;
                    it.hi = n;
                    it.clip = 0;
                }
                it.slots_log2 = (uint16_t)slots_for(min(kc, W.dp - kk * kc), kc);
                it.mask = 1u;
                items[out++] = it;
            }
        }
    }
}

// Three CTA shapes: T = 128 threads (8 CTAs per SM, a 16 KB region A:
// bitmaps over fewer than 131,072 ranks), T = 256 (4 CTAs per SM, 32 KB:
// 262,144 ranks) and T = 512 (2 CTAs per SM, 64 KB: 524,288 ranks).  Region A holds
// the bitmap or the table keys and masks (half of it each: 16T slots, so 8T
// keys per item); thread t owns words [32t, 32t + 32) of it in the bitmap
// prefix scan.
template <bool PV, int T>
__global__ void __launch_bounds__(T, 1024 / T)
    k_tc_hash(const HashGraph G, const VItem* __restrict__ items,
              uint32_t nitems, unsigned int* __restrict__ cursor, unsigned long long* __restrict__ partials,
              RunCtl* __restrict__ ctl) {
    extern __shared__ uint32_t hsm[];
    // Region A: the bitmap of a bitmap-mode item, the 16-bit rank entries of
    // a dense-mode item (ranges narrower than 2 x region A words), or the keys
    // and member masks of a hash-mode item; all zero between items.  Region B
    // (per-vertex counts only) holds 16-bit counters, two per word (a counter
    // counts at most one hit per in-edge of the item): in hash mode one per
    // table slot; in bitmap and dense mode one per key, indexed by the key's
    // rank in v's sorted list, after (bitmap mode) a 16-bit running popcount
    // per bitmap word.
    uint32_t* regA = hsm;
    constexpr int kHThreads = T, kHWarps = T / 32;
    constexpr uint32_t kRegionA = 32u * T;           // words
    constexpr uint32_t kBitmapBits = 32u * kRegionA;  // third-vertex ranges narrower than this: a bitmap
    constexpr uint32_t kMaxSlots = kRegionA / 2;     // table slots (keys, then member masks)
    constexpr uint32_t kDenseRanks = 2u * kRegionA;   // narrower ranges: 16-bit rank entries
    uint32_t* regB = hsm + kRegionA;
    __shared__ uint32_t s_wsum[kHWarps];
    __shared__ VItem s_it, s_itn;      // current item and the next one (prefetched)
    __shared__ unsigned long long s_cnt;
    __shared__ uint32_t s_item, s_itemn, s_vmask, s_next, s_rb, s_re, s_rbn, s_ren;
    __shared__ uint32_t s_edge[kHWarps][32];
    __shared__ uint32_t s_vcnt[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (uint32_t i = tid; i < kRegionA; i += kHThreads) regA[i] = 0;
    if (tid == 0) s_cnt = 0;
    if (PV) s_edge[warp][lane] = 0;
    // thread 0 fetches the next item, and a singleton's row bounds, ahead
    // into the second shared slot
    // every kStopCheckEvery-th fetch also reads the run's stop word; a stop
    // pushes the cursor past the end, so every CTA ends after its item
    auto prefetch = [&] {
        s_itemn = atomicAdd(cursor, 1u);
        if (s_itemn % kStopCheckEvery == 0 && s_itemn < nitems && run_stop_requested(ctl)) {
            atomicMax(cursor, nitems);
            s_itemn = nitems;
        }
        if (s_itemn < nitems) {
            const VItem nx = items[s_itemn];
            s_itn = nx;
            if (nx.nv == 1) {
                s_rbn = __ldg(G.rowptr + nx.v0);
                s_ren = __ldg(G.rowptr + nx.v0 + 1);
            }
        }
    };
    if (tid == 0) prefetch();
    unsigned long long cnt = 0;
    for (;;) {
        if (tid == 0) {
            s_item = s_itemn;
            s_it = s_itn;
            s_rb = s_rbn;
            s_re = s_ren;
            s_vmask = 0;
            s_next = 0;
        }
        if (PV && tid < 32) s_vcnt[tid] = 0;
        __syncthreads();
        if (s_item >= nitems) break;
        const VItem I = s_it;
        const bool single = I.nv == 1;
        // third-vertex range of the item: a singleton's partner entries all
        // exceed v, so its range starts at v + 1
        const uint32_t rlo = I.clip ? I.lo : (single ? I.v0 + 1 : 0);
        const uint32_t rhi = I.clip ? I.hi : G.n;
        // A bitmap or dense range is strictly narrower than region A holds,
        // so the slot just past it (at span) stays zero: a lookup of an
        // entry outside its in-edge's row reads that slot instead of taking
        // a branch.
        const bool bitmap = single && rhi - rlo < kBitmapBits;
        // a range narrower than kDenseRanks ranks (the top of the degree order:
        // most lookups at R-MAT scale) is held densely instead: one 16-bit
        // entry per rank, the key's rank in the list plus one (0: absent),
        // so a lookup is one shared load giving the hit and its counter
        const bool dense = bitmap && rhi - rlo < kDenseRanks;
        const uint32_t span = rhi - rlo;
        // a singleton's (clipped) list; its row bounds came with the item
        uint32_t rb = 0, re = 0;
        if (single) {
            rb = s_rb;
            re = s_re;
            if (I.clip) {
                rb = hlower_bound_b(G.col, G.vbase, rb, re, I.lo);
                re = hlower_bound_b(G.col, G.vbase, rb, re, I.hi);
            }
        }
        const uint32_t L = I.slots_log2, S = 1u << L;
        uint32_t* keys = regA;
        uint32_t* masks = regA + kMaxSlots;
        uint32_t* cnts = bitmap ? regB + kRegionA / 2 : regB;  // 16-bit counter i: half i & 1 of word i >> 1
        uint16_t* pre = reinterpret_cast<uint16_t*>(regB);
        uint16_t* dense16 = reinterpret_cast<uint16_t*>(regA);
        if (!bitmap)
            for (uint32_t i = tid; i < S; i += kHThreads) keys[i] = kEmpty;
        if (PV) {
            const uint32_t nc = bitmap ? re - rb : S;
            for (uint32_t i = tid; i < (nc + 1) / 2; i += kHThreads) cnts[i] = 0;
        }
        __syncthreads();
        // build: a singleton's list is inserted by the whole CTA (bitmap bits,
        // plus table keys for per-vertex counts); a group's members are
        // spread over the warps (member t to warp t mod kHWarps)
        if (single) {
            if (tid == 0 && rb < re) s_vmask = 1u;
            for (uint32_t q = rb + tid; q < re; q += kHThreads) {
                const uint32_t x = __ldg(G.col + (q - G.vbase));
                if (dense) dense16[x - rlo] = (uint16_t)(q - rb + 1);  // at most K keys: fits 16 bits
                else if (bitmap) atomicOr(&regA[(x - rlo) >> 5], 1u << ((x - rlo) & 31));
                else table_insert(keys, masks, x, 0u, L);
            }
        } else {
            for (uint32_t t = warp; t < I.nv; t += kHWarps) {
                const uint32_t v = I.v0 + t;
                // only members with in-edges in this item's index: the table
                // is sized for their lists alone
                if (!((I.mask >> t) & 1u)) continue;
                const uint32_t b = __ldg(G.rowptr + v), e = __ldg(G.rowptr + v + 1);
                if (b >= e) continue;
                const uint32_t bit = 1u << t;
                if (lane == 0) atomicOr(&s_vmask, bit);
                for (uint32_t q = b + lane; q < e; q += 32)
                    table_insert(keys, masks, __ldg(G.col + (q - G.vbase)), bit, L);
            }
        }
        __syncthreads();
        if (PV && bitmap && !dense) {
            // running popcount per bitmap word: thread t owns 32 consecutive
            // words; a CTA scan of the per-thread sums gives each its base
            const uint32_t nwords = (rhi - rlo + 31) >> 5;
            const uint32_t w0 = tid * 32;
            uint32_t own_sum = 0;
            for (uint32_t w = w0; w < w0 + 32 && w < nwords; ++w) own_sum += __popc(regA[w]);
            uint32_t inc = own_sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(kFullMask, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane == 31) s_wsum[warp] = inc;
            __syncthreads();
            uint32_t run = inc - own_sum;
            for (int w = 0; w < warp; ++w) run += s_wsum[w];
            for (uint32_t w = w0; w < w0 + 32 && w < nwords; ++w) {
                pre[w] = (uint16_t)run;
                run += __popc(regA[w]);
            }
            __syncthreads();
        }
        if (tid == 0) prefetch();
        const uint32_t vmask = s_vmask;
        // probe: warps take batches of 32 in-edges from a shared counter (so a
        // warp with short lists takes more batches).  In the 256- and
        // 512-thread shapes batch b is strided across the item (lane l takes
        // in-edge b + l * nb), so the lanes of a warp hold tails from all over
        // the item rather than 32 neighbouring ones (measured 2.6% faster at
        // R-MAT scale 24 with 256 threads, 3.5% at scale 27 with 512); the
        // 128-thread shape keeps 32 consecutive in-edges per batch (strided
        // was 3.4% slower at scale 23).
        // The probe loop, compiled once per lookup mode (the mode is fixed for
        // the item), so that no lookup tests it.
        auto probe = [&](auto mode) {
            constexpr int M = decltype(mode)::value;
            constexpr bool kStrided = T >= 256;
            const uint32_t nb = (I.in_end - I.in_begin + 31) >> 5;
            for (;;) {
                uint32_t b = 0;
                if (lane == 0) b = atomicAdd(&s_next, 1u);
                b = __shfl_sync(kFullMask, b, 0);
                if (b >= nb) break;
                const uint32_t idx = kStrided ? I.in_begin + b + lane * nb : I.in_begin + b * 32 + lane;
                uint32_t sb = 0, sl = 0, vbit = 0, e = 0;
                if (idx < I.in_end) {
                    const unsigned long long r = __ldg(G.xr + idx);
                    uint32_t xb = (uint32_t)r, xe = (uint32_t)(r >> 32);
                    e = xb - 1;
                    // a singleton item's in-edges all end at v0; a group's need
                    // the head read back to pick the member bit
                    const uint32_t v = single ? I.v0 : __ldg(G.colu + (e - G.ubase));
                    vbit = 1u << (v - I.v0);
                    if ((vmask & vbit) && e < G.core_e0) {
                        if (I.clip) {
                            xb = hlower_bound_b(G.colu, G.ubase, xb, xe, I.lo);
                            xe = hlower_bound_b(G.colu, G.ubase, xb, xe, I.hi);
                        }
                        sb = xb;
                        sl = xe - xb;
                    }
                }
                // The lists of the batch, cut into aligned 8-entry pairs of quads,
                // form one sequence that the lanes share: each lane takes
                // kPairSlots pairs per step with one 32-byte load each, so many
                // loads per lane are in flight across in-edge boundaries, and the
                // owner lookup is paid once per 8 entries.
                const uint32_t qa = sb >> 3;
                const uint32_t nq = sl ? ((sb + sl + 7) >> 3) - qa : 0;
                uint32_t incl = nq;
    #pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t y = __shfl_up_sync(kFullMask, incl, o);
                    if (lane >= o) incl += y;
                }
                const uint32_t total = __shfl_sync(kFullMask, incl, 31);
                const uint32_t excl = incl - nq;
                const uint32_t send = sb + sl;
                uint32_t tally = 0, tally_own = 0;  // per-vertex runs: this lane's hits for owner tally_own
                constexpr int U = kPairSlots;
                for (uint32_t r0 = 0; r0 < total; r0 += 32 * U) {
                    uint4 qv[U], qw[U];
                    uint32_t qb[U], lo_[U], hi_[U], bits[U], own[U];
    #pragma unroll
                    for (int j = 0; j < U; ++j) {
                        const uint32_t f = r0 + 32 * j + lane;
                        int o = 0;
    #pragma unroll
                        for (int step = 16; step >= 1; step >>= 1) {
                            uint32_t ex = __shfl_sync(kFullMask, excl, o + step);
                            if (ex <= f) o += step;
                        }
                        const uint32_t o_ex = __shfl_sync(kFullMask, excl, o);
                        lo_[j] = __shfl_sync(kFullMask, sb, o);
                        hi_[j] = __shfl_sync(kFullMask, send, o);
                        bits[j] = __shfl_sync(kFullMask, vbit, o);
                        own[j] = o;
                        qb[j] = 8 * ((lo_[j] >> 3) + (f - o_ex));
                        if (f < total) {
                            // one 256-bit read-only load per pair (32-byte aligned:
                            // qb and ubase are multiples of 8, colu is checked at launch)
                            const uint32_t* a = G.colu + (qb[j] - G.ubase);
                            asm("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                                : "=r"(qv[j].x), "=r"(qv[j].y), "=r"(qv[j].z), "=r"(qv[j].w), "=r"(qw[j].x),
                                  "=r"(qw[j].y), "=r"(qw[j].z), "=r"(qw[j].w)
                                : "l"(a));
                        } else {
                            qv[j] = qw[j] = make_uint4(kEmpty, kEmpty, kEmpty, kEmpty);
                        }
                        if (f >= total) hi_[j] = 0;
                    }
    #pragma unroll
                    for (int j = 0; j < U; ++j) {
                        const uint32_t xv[8] = {qv[j].x, qv[j].y, qv[j].z, qv[j].w, qw[j].x, qw[j].y, qw[j].z, qw[j].w};
                        uint32_t h4 = 0;
                        // entries of the pair inside the owner's range [lo, hi)
                        // as an 8-bit mask (qb > lo - 8 for every slot; a slot
                        // past the batch has hi = 0 and an empty mask)
                        const uint32_t va = lo_[j] > qb[j] ? lo_[j] - qb[j] : 0u;
                        const uint32_t vb = hi_[j] < qb[j] + 8 ? min(qb[j] + 8 - hi_[j], 8u) : 0u;
                        const uint32_t vm = (0xFFu << va) & (0xFFu >> vb);
    #pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const bool in = (vm >> i) & 1u;
                            if constexpr (M == kModeTable) {
                                if (!in) continue;
                            }
                            const uint32_t x = xv[i];
                            bool hit;
                            uint32_t h = 0;
                            if constexpr (M == kModeDense) {
                                // an entry outside the in-edge's row reads the zero slot at span
                                const uint32_t r1 = dense16[in ? x - rlo : span];
                                hit = r1 != 0u;
                                h = r1 - 1u;
                            } else if constexpr (M == kModeBitmap) {
                                const uint32_t d = in ? x - rlo : span;
                                const uint32_t word = regA[d >> 5];
                                hit = (word >> (d & 31)) & 1u;
                                // counter index = rank of x in v's sorted list
                                if (PV && hit) h = pre[d >> 5] + __popc(word & ((1u << (d & 31)) - 1u));
                            } else {
                                h = table_find(keys, x, L);
                                hit = h != kEmpty && (single || (masks[h] & bits[j]));
                            }
                            if (hit) {
                                ++h4;
                                if (PV) atomicAdd(&cnts[h >> 1], 1u << ((h & 1) << 4));
                            }
                        }
                        cnt += h4;
                        if (PV) {
                            // per-in-edge tally: a lane's slots belong to
                            // non-decreasing owners, so it sums its hits in a
                            // register and adds them to the owner's shared slot
                            // only when its owner changes
                            if (own[j] != tally_own) {
                                if (tally) atomicAdd(&s_edge[warp][tally_own], tally);
                                tally_own = own[j];
                                tally = 0;
                            }
                            tally += h4;
                        }
                    }
                }
                if (PV) {
                    if (tally) atomicAdd(&s_edge[warp][tally_own], tally);
                    __syncwarp();
                    const uint32_t c = s_edge[warp][lane];
                    if (c) {
                        s_edge[warp][lane] = 0;
                        // the tail u: from the streamed per-in-edge tails when the
                        // row index is not resident, else from the row index
                        const uint32_t u = G.itail ? __ldg(G.itail + idx) : __ldg(G.rowidx + e);
                        atomicAdd(G.tv + u, (unsigned long long)c);
                        atomicAdd(&s_vcnt[31 - __clz(vbit)], c);
                    }
                    __syncwarp();
                }
            }
        };
        if (dense) probe(std::integral_constant<int, kModeDense>{});
        else if (bitmap) probe(std::integral_constant<int, kModeBitmap>{});
        else probe(std::integral_constant<int, kModeTable>{});
        // the item's count goes to the CTA's shared accumulator
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(kFullMask, cnt, o);
        if (lane == 0 && cnt) atomicAdd(&s_cnt, cnt);
        cnt = 0;
        __syncthreads();
        if (PV) {
            if (bitmap) {
                // the key of rank i is the i-th entry of v's (clipped) list
                for (uint32_t i = tid; i < re - rb; i += kHThreads) {
                    const uint32_t c = (cnts[i >> 1] >> ((i & 1) << 4)) & 0xffffu;
                    if (c) atomicAdd(G.tv + __ldg(G.col + (rb + i - G.vbase)), (unsigned long long)c);
                }
            } else {
                for (uint32_t i = tid; i < S; i += kHThreads) {
                    const uint32_t c = (cnts[i >> 1] >> ((i & 1) << 4)) & 0xffffu;
                    if (c) atomicAdd(G.tv + keys[i], (unsigned long long)c);
                }
            }
            if (tid < I.nv && s_vcnt[tid]) atomicAdd(G.tv + I.v0 + tid, (unsigned long long)s_vcnt[tid]);
        }
        // leave region A all zero for the next item
        if (dense) {
            for (uint32_t q = rb + tid; q < re; q += kHThreads) dense16[__ldg(G.col + (q - G.vbase)) - rlo] = 0;
        } else if (bitmap) {
            for (uint32_t q = rb + tid; q < re; q += kHThreads) regA[(__ldg(G.col + (q - G.vbase)) - rlo) >> 5] = 0;
        } else {
            for (uint32_t i = tid; i < S; i += kHThreads) {
                regA[i] = 0;
                masks[i] = 0;
            }
        }
        __syncthreads();
    }
    // the CTA's total: partials[blockIdx.x]
    __syncthreads();
    if (tid == 0) partials[blockIdx.x] = s_cnt;
}

template <bool PV, int T>
size_t hash_smem() {
    // region B: max(16-bit slot counters, 16-bit word prefix + 16-bit per-key counters)
    constexpr uint32_t kRegionA = 32u * T, kMaxSlots = kRegionA / 2, kKeyCap = kMaxSlots / 2;
    constexpr uint32_t kRegionB =
        (kRegionA / 2 + kKeyCap / 2) > kMaxSlots / 2 ? (kRegionA / 2 + kKeyCap / 2) : kMaxSlots / 2;
    return (size_t)(kRegionA + (PV ? kRegionB : 0)) * sizeof(uint32_t);
}

template <bool PV, int T>
int grid_of() {
    int dev = 0, sms = 0, per_sm = 0;
    PGB_CUDA(cudaGetDevice(&dev));
    PGB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = hash_smem<PV, T>();
    PGB_CUDA(cudaFuncSetAttribute(k_tc_hash<PV, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PGB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tc_hash<PV, T>, T, smem));
    return std::max(1, per_sm) * sms;
}

template <bool PV, int T>
void launch_shape(const HashGraph& G, const VItem* items, uint32_t nitems, cudaStream_t s, unsigned int* cursor,
                  unsigned long long* partials, int grid, RunCtl* ctl) {
    k_tc_hash<PV, T><<<grid, T, hash_smem<PV, T>(), s>>>(G, items, nitems, cursor, partials, ctl);
}

}  // namespace

uint32_t build_hash_items_in(const ItemSpace& sp, uint32_t in_chunk, cudaStream_t s, DevBuf<VItem>& items) {
    if (in_chunk == 0) in_chunk = kInChunkDefault;
    in_chunk = std::min(in_chunk, kInChunkMax);
    const uint32_t nwin = sp.nwin;
    if (nwin == 0) {
        items.alloc(1, s);
        return 0;
    }
    DevBuf<uint32_t> counts((size_t)nwin + 1, s), offs((size_t)nwin + 1, s);
    PGB_CUDA(cudaMemsetAsync(counts.ptr + nwin, 0, 4, s));
    const int wgrid = (int)std::min<uint64_t>(((uint64_t)nwin * 32 + 255) / 256, 148ull * 64);
    k_items_count<<<wgrid, 256, 0, s>>>(sp, in_chunk, counts.ptr);
    PGB_CHECK_LAUNCH("k_items_count");
    Scratch scratch;
    size_t tmp = 0;
    PGB_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tmp, counts.ptr, offs.ptr, (int64_t)nwin + 1, s));
    void* t = scratch.get(tmp, s);
    PGB_CUDA(cub::DeviceScan::ExclusiveSum(t, tmp, counts.ptr, offs.ptr, (int64_t)nwin + 1, s));
    uint32_t nitems = 0;
    PGB_CUDA(cudaMemcpyAsync(&nitems, offs.ptr + nwin, 4, cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaStreamSynchronize(s));
    items.alloc(std::max<uint32_t>(nitems, 1), s);
    if (nitems) {
        k_items_emit<<<wgrid, 256, 0, s>>>(sp, in_chunk, offs.ptr, items.ptr);
        PGB_CHECK_LAUNCH("k_items_emit");
    }
    return nitems;
}

uint32_t build_hash_items(const pgb_blocks* b, uint32_t in_chunk, int threads, cudaStream_t s,
                          DevBuf<VItem>& items, const uint8_t* part_hash) {
    if (b->m == 0) {
        items.alloc(1, s);
        return 0;
    }
    ItemSpace sp{b->rowptr.ptr, b->colptr.ptr, b->col.ptr, 0, 0, 0, (b->n + 31) / 32, b->n,
                 key_capacity(threads), bitmap_range(threads)};
    if (part_hash) {
        sp.part_hash = part_hash;
        sp.cuts = b->cuts_d.ptr;
        sp.p = b->p;
    }
    return build_hash_items_in(sp, in_chunk, s, items);
}

HashGraph resident_hash_graph(const pgb_blocks* b, unsigned long long* tv) {
    HashGraph G{b->rowptr.ptr, b->col.ptr, b->rowidx.ptr, b->xr.ptr, tv, b->n};
    G.colu = b->col.ptr;
    return G;
}

int hash_threads(uint32_t n) { return n >= kWidestShapeVertices ? 512 : n >= kWideShapeVertices ? 256 : 128; }

int hash_grid(bool pv, int threads) {
    if (threads == 512) return pv ? grid_of<true, 512>() : grid_of<false, 512>();
    if (threads == 256) return pv ? grid_of<true, 256>() : grid_of<false, 256>();
    return pv ? grid_of<true, 128>() : grid_of<false, 128>();
}

void launch_hash(const HashGraph& G, const VItem* items, uint32_t nitems, bool pv, cudaStream_t s,
                 unsigned int* cursor, unsigned long long* partials, int grid, int threads, RunCtl* ctl) {
    // the pair loads read 32 aligned bytes at colu + (8k - ubase)
    if ((reinterpret_cast<uintptr_t>(G.colu) & 31) || (G.ubase & 7))
        fail(PGB_E_INVAL, "tail column view is not 32-byte aligned");
    PGB_CUDA(cudaMemsetAsync(cursor, 0, 4, s));
    if (threads == 512) {
        if (pv) launch_shape<true, 512>(G, items, nitems, s, cursor, partials, grid, ctl);
        else launch_shape<false, 512>(G, items, nitems, s, cursor, partials, grid, ctl);
    } else if (threads == 256) {
        if (pv) launch_shape<true, 256>(G, items, nitems, s, cursor, partials, grid, ctl);
        else launch_shape<false, 256>(G, items, nitems, s, cursor, partials, grid, ctl);
    } else {
        if (pv) launch_shape<true, 128>(G, items, nitems, s, cursor, partials, grid, ctl);
        else launch_shape<false, 128>(G, items, nitems, s, cursor, partials, grid, ctl);
    }
    PGB_CHECK_LAUNCH("k_tc_hash");
}

}  // namespace pgb
