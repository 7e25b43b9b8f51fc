// Triangle counting over block tuples (PGAbB Section 3.6, Listing 5)
// and its reduction (Section 3.3 reduce_dev).
//
// A block tuple is (A_ij, A_i[k0..k1], A_j[k0..k1]) with the third index a
// run of consecutive column blocks; k0 == k1 is the paper's block triple.
// For every oriented edge (u, v) of A_ij the kernel counts
//     | N+(u) ∩ N+(v) ∩ [lo, hi) |,   lo = c_k0, hi = c_(k1+1),
// where both partial lists are contiguous slices of the sorted rows (the
// parts are contiguous rank ranges).  Only entries of N+(u) after v can
// match (N+(v) holds ranks > v), so u's list starts right after v.
//
// Warp organisation (binary-search variant): 32 edges per warp step, one per
// lane.  Each lane picks the shorter of its two lists; a warp prefix sum
// flattens all (edge, element) work items of the 32 edges, so the warp's
// lanes stay busy whatever the list lengths.  Each item is looked up by
// binary search in the edge's longer list.  Counts stay in registers and are
// reduced per CTA into a per-CTA slot (no global atomics for the total).
#include <algorithm>
#include <memory>

#include "hybrid.cuh"
#include "core.cuh"
#include "internal.cuh"
#include "tc_hash.cuh"

namespace pgb {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

struct Tuple {
    uint32_t e_begin;  // first position in bedge
    uint32_t e_count;  // edges of A_ij covered
    uint32_t lo, hi;   // third-vertex rank range [lo, hi)
    uint32_t clip;     // 1 when lists must be clipped to [lo, hi)
    uint32_t variant;
};

struct Graph {
    // edge positions of a tuple's edges: bedge[idx] (block-grouped, PLAIN
    // mode), or, when xr is set, the in-edge index's (uint32)xr[idx] - 1
    // (grouped by head: the in-edges of a head part are one range)
    const uint32_t* __restrict__ bedge;
    const unsigned long long* __restrict__ xr;
    const uint32_t* __restrict__ rowidx;
    const uint32_t* __restrict__ col;
    const uint32_t* __restrict__ rowptr;
    unsigned long long* __restrict__ tv;  // per-vertex counts, rank space (may be null)
    // first CSR position of the dense top block's rows: an in-edge whose
    // tail row starts there or later has all three vertices of its
    // triangles in the block, which the dense count covers (core.cu)
    uint32_t core_e0 = 0xFFFFFFFFu;
};

__device__ __forceinline__ uint32_t edge_at(const Graph& G, uint32_t idx) {
    return G.xr ? (uint32_t)__ldg(G.xr + idx) - 1u : __ldg(G.bedge + idx);
}

__device__ __forceinline__ uint32_t lower_bound(const uint32_t* __restrict__ a, uint32_t b, uint32_t e,
                                                uint32_t x) {
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

// One warp step over up to 32 edges (lane `lane` owns bedge[idx] if valid).
template <bool PV>
__device__ __forceinline__ void warp_step(const Graph& G, uint32_t idx, bool valid, uint32_t lo, uint32_t hi,
                                          bool clip, unsigned long long& cnt, uint32_t* s_edge, int lane) {
    uint32_t sb = 0, sl = 0, lb = 0, ll = 0, u = 0, v = 0;
    const uint32_t e = valid ? edge_at(G, idx) : 0u;
    if (valid && e < G.core_e0) {
        u = __ldg(G.rowidx + e);
        v = __ldg(G.col + e);
        uint32_t xb = e + 1, xe = __ldg(G.rowptr + u + 1);
        uint32_t yb = __ldg(G.rowptr + v), ye = __ldg(G.rowptr + v + 1);
        if (clip) {
            xb = lower_bound(G.col, xb, xe, lo);
            xe = lower_bound(G.col, xb, xe, hi);
            yb = lower_bound(G.col, yb, ye, lo);
            ye = lower_bound(G.col, yb, ye, hi);
        }
        const uint32_t lx = xe - xb, ly = ye - yb;
        if (lx <= ly) {
            sb = xb; sl = lx; lb = yb; ll = ly;
        } else {
            sb = yb; sl = ly; lb = xb; ll = lx;
        }
        if (ll == 0) sl = 0;
    }
    uint32_t incl = sl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    const uint32_t excl = incl - sl;
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t f = base + lane;
        int o = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            uint32_t ex = __shfl_sync(kFull, excl, o + step);
            if (ex <= f) o += step;
        }
        const uint32_t o_ex = __shfl_sync(kFull, excl, o);
        const uint32_t o_sb = __shfl_sync(kFull, sb, o);
        const uint32_t o_lb = __shfl_sync(kFull, lb, o);
        const uint32_t o_ll = __shfl_sync(kFull, ll, o);
        if (f < total) {
            const uint32_t x = __ldg(G.col + o_sb + (f - o_ex));
            const uint32_t end = o_lb + o_ll;
            const uint32_t p = lower_bound(G.col, o_lb, end, x);
            if (p < end && __ldg(G.col + p) == x) {
                ++cnt;
                if (PV) {
                    atomicAdd(G.tv + x, 1ull);
                    atomicAdd(s_edge + o, 1u);
                }
            }
        }
    }
    if (PV) {
        __syncwarp();
        const uint32_t c = s_edge[lane];
        if (c) {
            atomicAdd(G.tv + u, (unsigned long long)c);
            atomicAdd(G.tv + v, (unsigned long long)c);
            s_edge[lane] = 0;
        }
        __syncwarp();
    }
}

// Warp-cooperative merge (PGB_VAR_MERGE) over up to 32 edges: the warp
// takes the lanes' edges one at a time and merges the two lists in chunks of
// 32 entries.  Each lane holds one entry of each chunk and finds its A entry
// among the B chunk with a 5-step shuffle search; the chunk whose last entry
// is smaller advances (both when equal).  A common entry is seen in exactly
// one step: once either chunk moves on, its entries cannot match later
// entries of the other list.
template <bool PV>
__device__ __forceinline__ void warp_step_merge(const Graph& G, uint32_t idx, bool valid, uint32_t lo, uint32_t hi,
                                                bool clip, unsigned long long& cnt, int lane) {
    uint32_t xb = 0, xe = 0, yb = 0, ye = 0, u = 0, v = 0;
    const uint32_t e = valid ? edge_at(G, idx) : 0u;
    if (valid && e < G.core_e0) {
        u = __ldg(G.rowidx + e);
        v = __ldg(G.col + e);
        xb = e + 1;
        xe = __ldg(G.rowptr + u + 1);
        yb = __ldg(G.rowptr + v);
        ye = __ldg(G.rowptr + v + 1);
        if (clip) {
            xb = lower_bound(G.col, xb, xe, lo);
            xe = lower_bound(G.col, xb, xe, hi);
            yb = lower_bound(G.col, yb, ye, lo);
            ye = lower_bound(G.col, yb, ye, hi);
        }
    }
    unsigned work = __ballot_sync(kFull, xb < xe && yb < ye);
    while (work) {
        const int j = __ffs(work) - 1;
        work &= work - 1;
        uint32_t pa = __shfl_sync(kFull, xb, j);
        const uint32_t ae = __shfl_sync(kFull, xe, j);
        uint32_t pb = __shfl_sync(kFull, yb, j);
        const uint32_t be = __shfl_sync(kFull, ye, j);
        uint32_t c = 0;
        while (pa < ae && pb < be) {
            const uint32_t na = min(32u, ae - pa), nb = min(32u, be - pb);
            const uint32_t av = (uint32_t)lane < na ? __ldg(G.col + pa + lane) : 0xffffffffu;
            const uint32_t bv = (uint32_t)lane < nb ? __ldg(G.col + pb + lane) : 0xffffffffu;
            const uint32_t amax = __shfl_sync(kFull, av, na - 1);
            const uint32_t bmax = __shfl_sync(kFull, bv, nb - 1);
            // first lane k of the B chunk with bv[k] >= av (31 if none)
            int k = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const uint32_t probe = __shfl_sync(kFull, bv, k + step - 1);
                if (probe < av) k += step;
            }
            const uint32_t at = __shfl_sync(kFull, bv, k);
            const bool hit = (uint32_t)lane < na && at == av;
            if (hit) {
                ++c;
                if (PV) atomicAdd(G.tv + av, 1ull);
            }
            if (amax <= bmax) pa += na;
            if (bmax <= amax) pb += nb;
        }
        cnt += c;
        if (PV) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(kFull, c, o);
            const uint32_t uj = __shfl_sync(kFull, u, j), vj = __shfl_sync(kFull, v, j);
            if (lane == 0 && c) {
                atomicAdd(G.tv + uj, (unsigned long long)c);
                atomicAdd(G.tv + vj, (unsigned long long)c);
            }
        }
    }
}

__device__ __forceinline__ void cta_reduce_store(unsigned long long cnt, unsigned long long* __restrict__ slot) {
    __shared__ unsigned long long s_red[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(kFull, cnt, o);
    if (lane == 0) s_red[warp] = cnt;
    __syncthreads();
    if (warp == 0) {
        cnt = lane < kWarps ? s_red[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(kFull, cnt, o);
        if (lane == 0) *slot = cnt;
    }
}

// PLAIN mode: one launch per block triple; warps stride over its edges.
template <bool PV>
__global__ void __launch_bounds__(kThreads)
    k_tc_tuple(Graph G, Tuple t, unsigned long long* __restrict__ partials, RunCtl* __restrict__ ctl) {
    __shared__ uint32_t s_edge[kWarps][32];
    __shared__ int s_stop;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // a stop request seen at entry skips the launch (its partial is 0)
    if (threadIdx.x == 0) s_stop = run_stop_requested(ctl) ? 1 : 0;
    __syncthreads();
    if (s_stop) {
        if (threadIdx.x == 0) partials[blockIdx.x] = 0;
        return;
    }
    if (PV) s_edge[warp][lane] = 0;
    __syncwarp();
    unsigned long long cnt = 0;
    const uint32_t gw = blockIdx.x * kWarps + warp, nw = gridDim.x * kWarps;
    const uint32_t end = t.e_begin + t.e_count;
    for (uint32_t i0 = t.e_begin + gw * 32; i0 < end; i0 += nw * 32) {
        const uint32_t idx = i0 + lane;
        if (t.variant == PGB_VAR_MERGE)
            warp_step_merge<PV>(G, idx, idx < end, t.lo, t.hi, t.clip != 0, cnt, lane);
        else
            warp_step<PV>(G, idx, idx < end, t.lo, t.hi, t.clip != 0, cnt, s_edge[warp], lane);
    }
    cta_reduce_store(cnt, partials + blockIdx.x);
}

// PERSISTENT mode: warps dequeue chunks of `chunk` edges from the tuple
// queue (chunk_prefix[t] = chunks before tuple t) with one atomic each.
template <bool PV>
__global__ void __launch_bounds__(kThreads)
    k_tc_persistent(Graph G, const Tuple* __restrict__ tuples, const uint32_t* __restrict__ chunk_prefix,
                    uint32_t ntuples, uint32_t chunk, unsigned int* __restrict__ cursor,
                    unsigned long long* __restrict__ partials, RunCtl* __restrict__ ctl) {
    __shared__ uint32_t s_edge[kWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (PV) s_edge[warp][lane] = 0;
    __syncwarp();
    const uint32_t total_chunks = chunk_prefix[ntuples];
    unsigned long long cnt = 0;
    while (true) {
        uint32_t c = 0;
        if (lane == 0) {
            c = atomicAdd(cursor, 1u);
            // every kStopCheckEvery-th chunk also reads the stop word; a stop
            // pushes the cursor past the end for every warp
            if (c % kStopCheckEvery == 0 && c < total_chunks && run_stop_requested(ctl)) {
                atomicMax(cursor, total_chunks);
                c = total_chunks;
            }
        }
        c = __shfl_sync(kFull, c, 0);
        if (c >= total_chunks) break;
        // tuple t: largest t with chunk_prefix[t] <= c
        uint32_t t = 0;
        if (lane == 0) {
            uint32_t lo = 0, hi = ntuples;
            while (hi - lo > 1) {
                uint32_t mid = (lo + hi) >> 1;
                if (__ldg(chunk_prefix + mid) <= c) lo = mid; else hi = mid;
            }
            t = lo;
        }
        t = __shfl_sync(kFull, t, 0);
        const Tuple tu = tuples[t];
        const uint32_t i0 = tu.e_begin + (c - __ldg(chunk_prefix + t)) * chunk;
        const uint32_t end = min(i0 + chunk, tu.e_begin + tu.e_count);
        for (uint32_t i = i0; i < end; i += 32) {
            const uint32_t idx = i + lane;
            if (tu.variant == PGB_VAR_MERGE)
                warp_step_merge<PV>(G, idx, idx < end, tu.lo, tu.hi, tu.clip != 0, cnt, lane);
            else
                warp_step<PV>(G, idx, idx < end, tu.lo, tu.hi, tu.clip != 0, cnt, s_edge[warp], lane);
        }
    }
    cta_reduce_store(cnt, partials + blockIdx.x);
}

// Sum of partials[0, n) into *out (one CTA).
__global__ void k_reduce_sum(const unsigned long long* __restrict__ partials, uint64_t n,
                             unsigned long long* __restrict__ out) {
    __shared__ unsigned long long s[32];
    unsigned long long acc = 0;
    for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kFull, acc, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        acc = lane < (int)(blockDim.x >> 5) ? s[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kFull, acc, o);
        if (lane == 0) *out = acc;
    }
}

// Per-segment sums: out[t] = sum partials[seg[t], seg[t+1]) (one CTA each).
__global__ void k_reduce_segments(const unsigned long long* __restrict__ partials, const uint64_t* __restrict__ seg,
                                  unsigned long long* __restrict__ out) {
    __shared__ unsigned long long s[32];
    const uint64_t b = seg[blockIdx.x], e = seg[blockIdx.x + 1];
    unsigned long long acc = 0;
    for (uint64_t i = b + threadIdx.x; i < e; i += blockDim.x) acc += partials[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kFull, acc, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        acc = lane < (int)(blockDim.x >> 5) ? s[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kFull, acc, o);
        if (lane == 0) out[blockIdx.x] = acc;
    }
}

// t[pairs[2i]] += pairs[2i + 1] for i < k (the host kernel's per-vertex
// counts, a vertex possibly in several pairs).
__global__ void k_add_pairs(unsigned long long* __restrict__ t, const uint32_t* __restrict__ pairs, uint64_t k) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride)
        atomicAdd(t + pairs[2 * i], (unsigned long long)pairs[2 * i + 1]);
}

// Rank-space per-vertex counts to original IDs.
__global__ void k_scatter_orig(const unsigned long long* __restrict__ tv, const uint32_t* __restrict__ perm,
                               uint32_t n, unsigned long long* __restrict__ out) {
    uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) out[perm[r]] = tv[r];
}

static int sm_count() {
    static int cached = 0;
    if (!cached) {
        int dev = 0;
        PGB_CUDA(cudaGetDevice(&dev));
        PGB_CUDA(cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev));
    }
    return cached;
}

}  // namespace pgb

struct pgb_tc_result {
    cudaStream_t stream = nullptr;
    uint32_t n = 0;
    bool per_vertex = false;
    bool per_triple = false;
    uint64_t ntriples = 0;
    int variant = PGB_VAR_BSEARCH;  // the variant that ran (PGB_VAR_MIXED: per part)
    std::vector<int32_t> part_variant;  // p: the kernel that counted each head part
    uint64_t streamed = 0;          // host-to-device bytes of a streamed run
    uint32_t chunks = 0;            // stream chunks (or pieces) of a streamed run (0 = resident)
    uint32_t slice_loads = 0;       // column slices copied in (column-streamed runs)
    uint32_t core_ranks = 0;        // ranks of the dense top block (0: none)
    pgb::DevBuf<unsigned long long> core_total;  // its triangles
    uint64_t core_lookups = 0;      // lookups it took off the intersection kernels
    double core_flop = 0;
    cudaEvent_t evc0 = nullptr, evc1 = nullptr;  // around its count (runs not replayed from a graph)
    pgb::DevBuf<unsigned long long> total;
    pgb::DevBuf<unsigned long long> tv_orig;
    pgb::DevBuf<unsigned long long> triple_counts;
    pgb::DevBuf<pgb::RunCtl> ctl;   // the run's stop word and its cancelled flag
    // HYBRID runs: the host kernel's share
    float host_ms = 0;
    uint64_t host_in_edges = 0;
    uint32_t host_parts = 0, host_threads = 0;
    bool host_cancelled = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    ~pgb_tc_result() {
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (evc0) cudaEventDestroy(evc0);
        if (evc1) cudaEventDestroy(evc1);
    }
};

namespace pgb {

static Tuple make_tuple(const pgb_blocks* b, uint32_t i, uint32_t j, uint32_t k0, uint32_t k1, int variant) {
    Tuple t;
    const size_t ij = (size_t)i * b->p + j;
    t.e_begin = (uint32_t)b->block_off[ij];
    t.e_count = (uint32_t)b->block_edges[ij];
    t.lo = b->cuts[k0];
    t.hi = b->cuts[k1 + 1];
    // v >= c_j and entries of both lists exceed v, so [c_j, n) needs no clipping
    t.clip = (t.lo > b->cuts[j] || t.hi < b->n) ? 1u : 0u;
    t.variant = (uint32_t)variant;
    return t;
}

// Autotuner.  The middle-vertex hash kernel pays a fixed cost per work item
// and wins when lists are long; the edge-wise binary-search kernel wins on
// flat graphs with short lists.  The statistic that separates them is the
// average number of lookups per oriented edge (the entries of the tail's row
// after the head): measured on one B300 the hash kernel is 5-10x faster on
// R-MAT (78-160 lookups per edge) and 1.6-18x slower on Erdos-Renyi (19),
// random geometric (1.5) and grid (0.55) graphs.
//
// The choice is made per column block j (head part V_j): an oriented edge
// (u, v) with v in V_j is the first edge of every triangle u < v < w it
// closes, so the tuples (A_ij, A_ik, A_jk) of one j, and the hash work items
// of the heads in V_j, count exactly the triangles whose middle vertex lies
// in V_j.  Each part takes the kernel its own lookups per edge favour, and
// both kernels add into the same counters.  A graph that mixes families (a
// serve batch is a disjoint union of R-MAT, grid and geometric jobs) gets
// the edge-wise kernel on its flat parts and the hash kernel on its skewed
// ones.
constexpr uint64_t kHashMinLookupsPerEdge = 32;

// Which kernel counts a head part (the triangles whose middle vertex lies in
// it): the edge-wise kernel, the hash kernel, or (HYBRID mode) the host.
enum : uint8_t { kPartEdge = 0, kPartHash = 1, kPartHost = 2 };

static uint64_t part_in_edges(const pgb_blocks* b, uint32_t j) {
    return b->head_off.size() > j + 1 ? b->head_off[j + 1] - b->head_off[j] : 0;
}

// Fills kind[j] for every head part and returns the device side's variant:
// PGB_VAR_BSEARCH, _MERGE or _HASH, or PGB_VAR_MIXED when parts with work
// go to both device kernels.
static int choose_variant(const pgb_blocks* b, const pgb_tc_opts& o, std::vector<uint8_t>& kind) {
    const uint32_t p = b->p;
    kind.assign(p, kPartEdge);
    std::vector<uint8_t> host(p, 0);
    if (o.mode == PGB_MODE_HYBRID) host = host_parts_by_cutoff(b, o.host_share_ppm ? o.host_share_ppm : 1000);
    int v;
    if (o.mode == PGB_MODE_PLAIN) v = o.variant == PGB_VAR_MERGE ? PGB_VAR_MERGE : PGB_VAR_BSEARCH;
    else if (b->offloaded) v = PGB_VAR_HASH;  // only the hash kernel reads a streamed index
    else v = o.variant;
    bool hash_work = false, edge_work = false;
    for (uint32_t j = 0; j < p; ++j) {
        if (host[j]) {
            kind[j] = kPartHost;
            continue;
        }
        if (v == PGB_VAR_HASH) {
            kind[j] = kPartHash;
        } else if (v == PGB_VAR_AUTO) {
            uint64_t edges = 0;
            for (uint32_t i = 0; i <= j; ++i) edges += b->block_edges[(size_t)i * p + j];
            const uint64_t probes = j < b->part_probes.size() ? b->part_probes[j] : 0;
            const uint64_t thr = o.hash_min_lookups ? o.hash_min_lookups : kHashMinLookupsPerEdge;
            kind[j] = (edges == 0 || probes >= thr * edges) ? kPartHash : kPartEdge;
        }
        const bool work = part_in_edges(b, j) > 0;
        hash_work |= work && kind[j] == kPartHash;
        edge_work |= work && kind[j] == kPartEdge;
    }
    if (v != PGB_VAR_AUTO) return v;
    if (hash_work && edge_work) return PGB_VAR_MIXED;
    return hash_work ? PGB_VAR_HASH : PGB_VAR_BSEARCH;
}

// Everything the device work of one run needs, allocated and planned before
// any of it is enqueued, so that the work can also be captured once in a
// CUDA graph and replayed (use_graph).
struct RunPlan {
    // settings the plan was made for
    int mode = 0, variant = 0, order = 0;
    bool per_vertex = false, per_triple = false;
    uint32_t chunk_edges = 0, hash_threads_opt = 0;
    uint32_t n = 0;
    DevBuf<unsigned long long> tv, partials, total, tv_orig, triple_counts;
    uint64_t npartials = 0;
    Graph G{};
    // PLAIN: one launch per block triple
    std::vector<Tuple> tuples;
    std::vector<int> grids;
    std::vector<uint64_t> seg;
    std::vector<uint32_t> launch_order;  // queue entries in launch order
    DevBuf<uint64_t> dseg;
    // PERSISTENT binary search: tuples drained from a device counter
    DevBuf<Tuple> dt;
    DevBuf<uint32_t> dcp;
    uint32_t nt = 0, chunk = 0;
    // PERSISTENT hash: work items (MIXED: those of the hash parts only)
    DevBuf<VItem> items;
    uint32_t nitems = 0;
    HashGraph H{};
    DevBuf<unsigned int> cursor;  // [0]: hash items, [1]: edge-wise chunks
    int grid = 0, threads = 128;
    int hgrid = 0;                // general plans: CTAs of the hash launch (partials [0, hgrid))
    bool general = false;         // parts split between kernels (and the host): filtered launches
    bool host_slot = false;       // HYBRID: partials[host_idx] holds the host's total
    uint64_t host_idx = 0;
    std::vector<uint8_t> part_kind;
    DevBuf<uint8_t> dpart_hash;
    const uint32_t* perm = nullptr;
    // per-part runs with both kernels: the edge-wise launch on a side
    // stream (forked and joined by events), so that it fills the SMs the
    // hash launch's last CTAs leave idle
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    // graph replay: the captured kernels read this plan-owned control block,
    // which each replay refills with the run's stop word
    DevBuf<RunCtl> ctl;
    // dense top block (core.cu): its plan, and its total in partials[core_slot]
    CorePlan core;
    uint64_t core_slot = 0;
    cudaGraphExec_t exec = nullptr;
    uint64_t graph_launches = 0;  // kernel launches one replay makes
    cudaEvent_t done = nullptr;   // the last replay's outputs have been copied out
    bool used = false;

    bool same(const pgb_tc_opts& o, int var, const std::vector<uint8_t>& kinds, uint32_t core_k) const {
        return mode == o.mode && variant == var && part_kind == kinds && order == o.order && core.K == core_k &&
               per_vertex == (o.per_vertex != 0) &&
               per_triple == (o.mode == PGB_MODE_PLAIN && o.per_triple != 0) && chunk_edges == o.chunk_edges &&
               hash_threads_opt == o.hash_threads;
    }
    ~RunPlan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (done) cudaEventDestroy(done);
        if (fork_ev) cudaEventDestroy(fork_ev);
        if (join_ev) cudaEventDestroy(join_ev);
        if (side) cudaStreamDestroy(side);
    }
};

static std::unique_ptr<RunPlan> prepare(const pgb_blocks* b, const pgb_tc_opts& o, int variant,
                                        const std::vector<uint8_t>& part_kind, uint32_t core_k, cudaStream_t s) {
    std::unique_ptr<RunPlan> P(new RunPlan());
    P->part_kind = part_kind;
    bool all_hash = true, any_host = false;
    for (uint8_t k : part_kind) {
        all_hash &= k == kPartHash;
        any_host |= k == kPartHost;
    }
    P->mode = o.mode;
    P->variant = variant;
    P->order = o.order;
    P->per_vertex = o.per_vertex != 0;
    P->per_triple = o.mode == PGB_MODE_PLAIN && o.per_triple != 0;
    P->chunk_edges = o.chunk_edges;
    P->hash_threads_opt = o.hash_threads;
    const uint32_t n = P->n = b->n;
    P->perm = b->perm.ptr;
    P->total.alloc(1, s);
    if (P->per_vertex) {
        P->tv.alloc(n, s);
        P->tv_orig.alloc(n, s);
    }
    // PLAIN launches walk the edges of one block A_ij (block-grouped index);
    // the persistent edge-wise kernel walks head parts of the in-edge index
    if (o.mode == PGB_MODE_PLAIN) {
        ensure_block_edge_index(b, s);
        P->G = Graph{b->bedge.ptr, nullptr, b->rowidx.ptr, b->col.ptr, b->rowptr.ptr, P->tv.ptr};
    } else {
        P->G = Graph{nullptr, b->xr.ptr, b->rowidx.ptr, b->col.ptr, b->rowptr.ptr, P->tv.ptr};
    }

    if (o.mode == PGB_MODE_PLAIN) {
        // one launch per block triple, in queue order
        const uint64_t T = b->triples.size();
        P->seg.assign(T + 1, 0);
        P->grids.resize(T);
        P->tuples.resize(T);
        for (uint64_t t = 0; t < T; ++t) {
            const pgb_triple& q = b->triples[t];
            uint64_t e = b->block_edges[(size_t)q.i * b->p + q.j];
            uint64_t g = (e + 32 * kWarps - 1) / (32 * kWarps);
            g = std::min<uint64_t>(std::max<uint64_t>(g, 1), (uint64_t)sm_count() * 8);
            P->grids[t] = (int)g;
            P->seg[t + 1] = P->seg[t] + g;
            P->tuples[t] = make_tuple(b, q.i, q.j, q.k, q.k, variant);
        }
        P->npartials = P->seg[T];
        P->partials.alloc(std::max<uint64_t>(P->npartials, 1), s);
        // launch order: the queue's, or along the Hilbert curve of the
        // blocks (i, j), then k; partials stay indexed by queue entry
        P->launch_order.resize(T);
        for (uint64_t t = 0; t < T; ++t) P->launch_order[t] = (uint32_t)t;
        if (o.order == PGB_ORDER_HILBERT && T > 1) {
            const std::vector<uint32_t> hb = hilbert_block_order(b->p);
            std::vector<uint32_t> pos((size_t)b->p * b->p, 0);
            for (size_t r = 0; r < hb.size(); ++r) pos[hb[r]] = (uint32_t)r;
            std::stable_sort(P->launch_order.begin(), P->launch_order.end(), [&](uint32_t x, uint32_t y) {
                const pgb_triple &a = b->triples[x], &c = b->triples[y];
                const uint32_t pa = pos[(size_t)a.i * b->p + a.j], pc = pos[(size_t)c.i * b->p + c.j];
                if (pa != pc) return pa < pc;
                return a.k < c.k;
            });
        }
        if (P->per_triple && T > 0) {
            P->dseg.alloc(T + 1, s);
            PGB_CUDA(cudaMemcpyAsync(P->dseg.ptr, P->seg.data(), (T + 1) * 8, cudaMemcpyHostToDevice, s));
            P->triple_counts.alloc(T, s);
        }
    } else if (variant == PGB_VAR_HASH && all_hash) {
        // middle-vertex hash variant over every head (tc_hash.cu)
        P->threads = o.hash_threads ? (int)o.hash_threads : hash_threads(b->n);
        P->nitems = build_hash_items(b, o.chunk_edges ? o.chunk_edges : kResidentInChunk, P->threads, s, P->items);
        if (P->nitems) {
            P->H = resident_hash_graph(b, P->tv.ptr);
            P->cursor.alloc(2, s);
            P->grid = hash_grid(P->per_vertex, P->threads);
            P->npartials = (uint64_t)P->grid;
            P->partials.alloc(P->npartials, s);
        }
    } else {
        // one tuple per head part j: the in-edges (u, v) with v in V_j, i.e.
        // the block column A_*j with third range [c_j, n) (the tuples
        // (A_ij, A_i[j..p-1], A_j[j..p-1]) of every i <= j), ordered by the
        // summed weight of its triples (ORDER_LOCALITY: by j, descending)
        // (head parts of the other kinds are left to the hash kernel or the host)
        const uint32_t p = b->p;
        P->general = true;
        P->host_slot = any_host;
        std::vector<uint64_t> w(p, 0);
        for (const pgb_triple& q : b->triples) w[q.j] += q.w;
        std::vector<uint32_t> ids;
        for (uint32_t j = 0; j < p; ++j)
            if (w[j] && b->head_off[j + 1] > b->head_off[j] && P->part_kind[j] == kPartEdge) ids.push_back(j);
        if (o.order == PGB_ORDER_LOCALITY)
            std::stable_sort(ids.begin(), ids.end(), [&](uint32_t x, uint32_t y) { return x > y; });
        else
            std::stable_sort(ids.begin(), ids.end(), [&](uint32_t x, uint32_t y) { return w[x] > w[y]; });
        const uint32_t chunk = P->chunk = o.chunk_edges ? ((o.chunk_edges + 31) / 32) * 32 : 64;
        std::vector<Tuple> tuples;
        std::vector<uint32_t> cp(1, 0);
        const int tvar = variant == PGB_VAR_MERGE ? PGB_VAR_MERGE : PGB_VAR_BSEARCH;
        for (uint32_t j : ids) {
            Tuple tu;
            tu.e_begin = (uint32_t)b->head_off[j];
            tu.e_count = (uint32_t)(b->head_off[j + 1] - b->head_off[j]);
            tu.lo = b->cuts[j];
            tu.hi = b->n;
            tu.clip = 0;  // every entry of both lists exceeds v >= c_j
            tu.variant = (uint32_t)tvar;
            tuples.push_back(tu);
            cp.push_back(cp.back() + (tu.e_count + chunk - 1) / chunk);
        }
        const uint32_t nt = P->nt = (uint32_t)tuples.size();
        P->dt.alloc(std::max<uint32_t>(nt, 1), s);
        P->dcp.alloc(cp.size(), s);
        P->cursor.alloc(2, s);
        if (nt) PGB_CUDA(cudaMemcpyAsync(P->dt.ptr, tuples.data(), nt * sizeof(Tuple), cudaMemcpyHostToDevice, s));
        PGB_CUDA(cudaMemcpyAsync(P->dcp.ptr, cp.data(), cp.size() * 4, cudaMemcpyHostToDevice, s));
        int per_sm = 0;
        if (P->per_vertex)
            PGB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tc_persistent<true>, kThreads, 0));
        else
            PGB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tc_persistent<false>, kThreads, 0));
        P->grid = std::max(1, per_sm) * sm_count();
        P->npartials = (uint64_t)P->grid;
        bool hash_parts = false;
        for (uint32_t j = 0; j < p; ++j) hash_parts |= P->part_kind[j] == kPartHash && b->head_off[j + 1] > b->head_off[j];
        if (hash_parts) {
            // the hash parts' items, counted by a hash launch before the
            // edge-wise one; its per-CTA totals come first in partials
            std::vector<uint8_t> mask(p);
            for (uint32_t j = 0; j < p; ++j) mask[j] = P->part_kind[j] == kPartHash ? 1 : 0;
            P->dpart_hash.alloc(p, s);
            PGB_CUDA(cudaMemcpyAsync(P->dpart_hash.ptr, mask.data(), p, cudaMemcpyHostToDevice, s));
            P->threads = o.hash_threads ? (int)o.hash_threads : hash_threads(b->n);
            P->nitems = build_hash_items(b, o.chunk_edges ? o.chunk_edges : kResidentInChunk, P->threads, s,
                                         P->items, P->dpart_hash.ptr);
            if (P->nitems) {
                P->H = resident_hash_graph(b, P->tv.ptr);
                P->hgrid = hash_grid(P->per_vertex, P->threads);
                P->npartials += (uint64_t)P->hgrid;
            }
        }
        if (P->nitems && P->hgrid && P->nt) {
            PGB_CUDA(cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking));
            PGB_CUDA(cudaEventCreateWithFlags(&P->fork_ev, cudaEventDisableTiming));
            PGB_CUDA(cudaEventCreateWithFlags(&P->join_ev, cudaEventDisableTiming));
        }
        if (P->host_slot) P->host_idx = P->npartials++;  // written once the host parts are counted
        P->partials.alloc(P->npartials, s);
        if (P->host_slot) PGB_CUDA(cudaMemsetAsync(P->partials.ptr + P->host_idx, 0, 8, s));
    }
    // the dense top block: the intersection kernels skip the in-edges whose
    // tail row starts at or after its first CSR position; its total takes one
    // more partial
    if (core_k) {
        core_prepare(b, core_k, s, P->core);
        P->G.core_e0 = P->core.e0;
        P->H.core_e0 = P->core.e0;
        P->core_slot = P->npartials;
        P->npartials += 1;
        P->partials.alloc(P->npartials, s);
        if (P->host_slot) PGB_CUDA(cudaMemsetAsync(P->partials.ptr + P->host_idx, 0, 8, s));
    }
    // the host arrays copied above are pageable; their copies are staged
    // before the calls return, so the vectors may change afterwards
    return P;
}

// The device work of a planned run: counters cleared, counting launches
// (between ev0 and ev1 when given), reductions.  Makes no allocation and no
// synchronising call, so it can be captured.
static void enqueue_reduce(const RunPlan& P, cudaStream_t s);

// The device work of a planned run: the counting launches (between ev0 and
// ev1 when given), then the reductions.
static void enqueue_count(const RunPlan& P, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, RunCtl* ctl,
                          cudaEvent_t evc0 = nullptr, cudaEvent_t evc1 = nullptr);

static void enqueue(const RunPlan& P, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, RunCtl* ctl,
                    cudaEvent_t evc0 = nullptr, cudaEvent_t evc1 = nullptr) {
    enqueue_count(P, s, ev0, ev1, ctl, evc0, evc1);
    enqueue_reduce(P, s);
}

static void enqueue_count(const RunPlan& P, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, RunCtl* ctl,
                          cudaEvent_t evc0, cudaEvent_t evc1) {
    if (P.per_vertex && P.n) PGB_CUDA(cudaMemsetAsync(P.tv.ptr, 0, (size_t)P.n * 8, s));
    if (ev0) PGB_CUDA(cudaEventRecord(ev0, s));
    if (P.mode == PGB_MODE_PLAIN) {
        const uint64_t T = P.tuples.size();
        for (uint64_t r = 0; r < T; ++r) {
            const uint32_t t = P.launch_order[r];
            if (P.per_vertex)
                k_tc_tuple<true><<<P.grids[t], kThreads, 0, s>>>(P.G, P.tuples[t], P.partials.ptr + P.seg[t], ctl);
            else
                k_tc_tuple<false><<<P.grids[t], kThreads, 0, s>>>(P.G, P.tuples[t], P.partials.ptr + P.seg[t], ctl);
        }
        PGB_CHECK_LAUNCHES("k_tc_tuple", T);
    } else if (!P.general) {
        if (P.nitems)
            launch_hash(P.H, P.items.ptr, P.nitems, P.per_vertex, s, P.cursor.ptr, P.partials.ptr, P.grid,
                        P.threads, ctl);
    } else {
        // the hash parts (their totals in partials [0, hgrid)) and the
        // edge-wise tuples of the edge-wise parts; with both, the edge-wise
        // launch runs on the side stream, beside the hash launch's tail
        unsigned int* bcur = P.cursor.ptr + 1;
        unsigned long long* bpart = P.partials.ptr + P.hgrid;
        PGB_CUDA(cudaMemsetAsync(bcur, 0, 4, s));
        const bool fork = P.side != nullptr;
        if (fork) {
            PGB_CUDA(cudaEventRecord(P.fork_ev, s));
            PGB_CUDA(cudaStreamWaitEvent(P.side, P.fork_ev, 0));
        }
        if (P.nitems && P.hgrid)
            launch_hash(P.H, P.items.ptr, P.nitems, P.per_vertex, s, P.cursor.ptr, P.partials.ptr, P.hgrid,
                        P.threads, ctl);
        const cudaStream_t es = fork ? P.side : s;
        if (P.per_vertex)
            k_tc_persistent<true><<<P.grid, kThreads, 0, es>>>(P.G, P.dt.ptr, P.dcp.ptr, P.nt, P.chunk, bcur, bpart,
                                                              ctl);
        else
            k_tc_persistent<false><<<P.grid, kThreads, 0, es>>>(P.G, P.dt.ptr, P.dcp.ptr, P.nt, P.chunk, bcur,
                                                               bpart, ctl);
        PGB_CHECK_LAUNCH("k_tc_persistent");
        if (fork) {
            PGB_CUDA(cudaEventRecord(P.join_ev, P.side));
            PGB_CUDA(cudaStreamWaitEvent(s, P.join_ev, 0));
        }
    }
    if (P.core.K) {
        if (evc0) PGB_CUDA(cudaEventRecord(evc0, s));
        core_enqueue(P.core, P.per_vertex ? P.tv.ptr : nullptr, P.partials.ptr + P.core_slot, s);
        if (evc1) PGB_CUDA(cudaEventRecord(evc1, s));
    }
    if (ev1) PGB_CUDA(cudaEventRecord(ev1, s));
}

static void enqueue_reduce(const RunPlan& P, cudaStream_t s) {
    if (P.per_triple && !P.tuples.empty()) {
        k_reduce_segments<<<(unsigned)P.tuples.size(), 256, 0, s>>>(P.partials.ptr, P.dseg.ptr, P.triple_counts.ptr);
        PGB_CHECK_LAUNCH("k_reduce_segments");
    }
    if (P.npartials)
        k_reduce_sum<<<1, 1024, 0, s>>>(P.partials.ptr, P.npartials, P.total.ptr);
    else
        PGB_CUDA(cudaMemsetAsync(P.total.ptr, 0, 8, s));
    PGB_CHECK_LAUNCH("k_reduce_sum");
    if (P.per_vertex && P.n) {
        k_scatter_orig<<<std::min<uint32_t>((P.n + 255) / 256, 148 * 32), 256, 0, s>>>(P.tv.ptr, P.perm, P.n,
                                                                                      P.tv_orig.ptr);
        PGB_CHECK_LAUNCH("k_scatter_orig");
    }
}

// Capture the plan's device work on a private stream and instantiate it.
static void capture(RunPlan& P) {
    cudaStream_t cs = nullptr;
    PGB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    uint64_t launches = 0;
    int rc = guard([&] {
        begin_launch_capture(&launches);
        PGB_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        int rc2 = guard([&] { enqueue(P, cs, nullptr, nullptr, P.ctl.ptr); });
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        end_launch_capture();
        if (rc2 != PGB_OK) fail(rc2, pgb_last_error());
        PGB_CUDA(e);
        PGB_CUDA(cudaGraphInstantiate(&P.exec, g, 0));
        PGB_CUDA(cudaEventCreateWithFlags(&P.done, cudaEventDisableTiming));
    });
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (rc != PGB_OK) fail(rc, pgb_last_error());
    P.graph_launches = launches;
}

static void run(const pgb_blocks* b, const pgb_tc_opts& o_in, cudaStream_t s, pgb_tc_result* r) {
    pgb_tc_opts o = o_in;
    std::vector<uint8_t> part_kind;
    o.variant = choose_variant(b, o_in, part_kind);
    r->variant = o.variant;
    r->part_variant.resize(b->p);
    for (uint32_t j = 0; j < b->p; ++j)
        r->part_variant[j] = part_kind[j] == kPartHost   ? PGB_VAR_HOST
                             : part_kind[j] == kPartHash ? PGB_VAR_HASH
                             : (o.variant == PGB_VAR_MERGE ? PGB_VAR_MERGE : PGB_VAR_BSEARCH);
    const uint32_t n = b->n;
    r->stream = s;
    r->n = n;
    r->per_vertex = o.per_vertex != 0;
    r->per_triple = o.mode == PGB_MODE_PLAIN && o.per_triple != 0;
    r->ntriples = b->triples.size();
    PGB_CUDA(cudaEventCreate(&r->ev0));
    PGB_CUDA(cudaEventCreate(&r->ev1));
    // the control block: the token's mapped word (or null), not cancelled;
    // staged from the stack (a pageable copy returns once staged)
    const RunCtl hctl{o.cancel ? o.cancel->dev : nullptr, 0u, 0u};
    r->ctl.alloc(1, s);
    PGB_CUDA(cudaMemcpyAsync(r->ctl.ptr, &hctl, sizeof(RunCtl), cudaMemcpyHostToDevice, s));

    if (b->offloaded) {
        // in-edge index in pinned host memory, streamed in chunks (stream.cu)
        r->total.alloc(1, s);
        DevBuf<unsigned long long> tv, partials;
        uint64_t npartials = 0;
        if (r->per_vertex) {
            tv.alloc(n, s);
            if (n) PGB_CUDA(cudaMemsetAsync(tv.ptr, 0, (size_t)n * 8, s));
        }
        // the index tier (rows and columns resident) takes the dense top block
        // too, its bytes charged to the device budget before the slots
        CorePlan core;
        uint64_t budget = o.device_budget;
        if (!b->cols_offloaded && (o_in.dense_core > 0 || (o_in.dense_core == 0 && o_in.variant == PGB_VAR_AUTO))) {
            const uint32_t k = choose_core(b, o_in.dense_core);
            const uint64_t need = k ? core_bytes(k) : 0;
            // at most half the budget goes to the block; the rest keeps the slots
            if (k && (budget == 0 || need <= budget / 2)) {
                core_prepare(b, k, s, core);
                if (budget) budget -= need;
                r->core_ranks = k;
                r->core_flop = core_flop(k);
                if (k % kCoreBand == 0)
                    for (uint32_t i = 0; i < k / kCoreBand && i < b->core_probes.size(); ++i)
                        r->core_lookups += b->core_probes[i];
            }
        }
        if (b->cols_offloaded)
            run_column_streaming(b, r->per_vertex, o.hash_threads, tv.ptr, o.device_budget, s, partials, npartials,
                                 r->ev0, r->ev1, &r->streamed, &r->chunks, &r->slice_loads, r->ctl.ptr);
        else
            run_streaming(b, o.chunk_edges, r->per_vertex, o.hash_threads, tv.ptr, budget, s, partials,
                          npartials, r->ev0, r->ev1, &r->streamed, &r->chunks, r->ctl.ptr,
                          core.K ? core.e0 : 0xFFFFFFFFu);
        if (npartials)
            k_reduce_sum<<<1, 1024, 0, s>>>(partials.ptr, npartials, r->total.ptr);
        else
            PGB_CUDA(cudaMemsetAsync(r->total.ptr, 0, 8, s));
        PGB_CHECK_LAUNCH("k_reduce_sum");
        if (core.K) {
            // after the streamed launches (run_streaming returned once they
            // completed); the count phase's end event moves past the block
            PGB_CUDA(cudaEventCreate(&r->evc0));
            PGB_CUDA(cudaEventCreate(&r->evc1));
            r->core_total.alloc(1, s);
            PGB_CUDA(cudaEventRecord(r->evc0, s));
            core_enqueue(core, r->per_vertex ? tv.ptr : nullptr, r->core_total.ptr, s);
            PGB_CUDA(cudaEventRecord(r->evc1, s));
            core_add_total(r->core_total.ptr, r->total.ptr, s);
            PGB_CUDA(cudaEventRecord(r->ev1, s));
        }
        if (r->per_vertex) {
            r->tv_orig.alloc(n, s);
            if (n) {
                k_scatter_orig<<<std::min<uint32_t>((n + 255) / 256, 148 * 32), 256, 0, s>>>(tv.ptr, b->perm.ptr, n,
                                                                                          r->tv_orig.ptr);
                PGB_CHECK_LAUNCH("k_scatter_orig");
            }
        }
        return;
    }
    // the dense top block: persistent runs with the autotuner, or asked for
    const uint32_t core_k =
        (o.mode == PGB_MODE_PERSISTENT || o.mode == PGB_MODE_HYBRID) &&
                (o_in.dense_core > 0 || (o_in.dense_core == 0 && o_in.variant == PGB_VAR_AUTO))
            ? choose_core(b, o_in.dense_core)
            : 0;
    r->core_ranks = core_k;
    if (core_k) {
        r->core_flop = core_flop(core_k);
        if (core_k % kCoreBand == 0)
            for (uint32_t i = 0; i < core_k / kCoreBand && i < b->core_probes.size(); ++i)
                r->core_lookups += b->core_probes[i];
    }
    auto keep_core_total = [&](const RunPlan& Q) {
        if (!core_k) return;
        r->core_total.alloc(1, s);
        PGB_CUDA(cudaMemcpyAsync(r->core_total.ptr, Q.partials.ptr + Q.core_slot, 8, cudaMemcpyDeviceToDevice, s));
    };
    if (o.mode == PGB_MODE_HYBRID) {
        // the device parts' launches are queued first; the host threads count
        // the host parts meanwhile; their total fills the plan's last partial
        // and their per-vertex counts are added before the reductions
        std::unique_ptr<RunPlan> P = prepare(b, o, o.variant, part_kind, core_k, s);
        if (core_k) {
            PGB_CUDA(cudaEventCreate(&r->evc0));
            PGB_CUDA(cudaEventCreate(&r->evc1));
        }
        enqueue_count(*P, s, r->ev0, r->ev1, r->ctl.ptr, r->evc0, r->evc1);
        keep_core_total(*P);
        std::vector<uint8_t> host_mask(b->p);
        for (uint32_t j = 0; j < b->p; ++j) host_mask[j] = part_kind[j] == kPartHost ? 1 : 0;
        std::vector<std::pair<uint32_t, uint32_t>> adds;
        // the host kernel skips the dense block's in-edges as the device kernels do
        const HostCountResult hr = host_count_parts(b, host_mask, o.host_threads, r->per_vertex, adds, o.cancel, s,
                                                    core_k ? P->core.e0 : 0xFFFFFFFFu);
        r->host_ms = hr.ms;
        r->host_in_edges = hr.in_edges;
        r->host_parts = hr.parts;
        r->host_threads = hr.threads;
        r->host_cancelled = hr.cancelled;
        if (P->host_slot) {
            const unsigned long long h_total = hr.total;
            PGB_CUDA(cudaMemcpyAsync(P->partials.ptr + P->host_idx, &h_total, 8, cudaMemcpyHostToDevice, s));
        }
        DevBuf<uint32_t> dadds;
        if (r->per_vertex && !adds.empty()) {
            // (vertex, count) pairs, staged from pageable memory
            dadds.alloc(2 * adds.size(), s);
            PGB_CUDA(cudaMemcpyAsync(dadds.ptr, adds.data(), adds.size() * 8, cudaMemcpyHostToDevice, s));
            const uint64_t k = adds.size();
            k_add_pairs<<<(unsigned)std::min<uint64_t>((k + 255) / 256, 148ull * 32), 256, 0, s>>>(P->tv.ptr,
                                                                                                  dadds.ptr, k);
            PGB_CHECK_LAUNCH("k_add_pairs");
        }
        enqueue_reduce(*P, s);
        // the host buffer is pageable: the copies above were staged before
        // returning, so it may go out of scope
        r->total = std::move(P->total);
        r->tv_orig = std::move(P->tv_orig);
        return;
    }
    if (!o.use_graph) {
        std::unique_ptr<RunPlan> P = prepare(b, o, o.variant, part_kind, core_k, s);
        if (core_k) {
            PGB_CUDA(cudaEventCreate(&r->evc0));
            PGB_CUDA(cudaEventCreate(&r->evc1));
        }
        enqueue(*P, s, r->ev0, r->ev1, r->ctl.ptr, r->evc0, r->evc1);
        keep_core_total(*P);
        // the outputs move to the result; the rest is released in stream order
        r->total = std::move(P->total);
        r->tv_orig = std::move(P->tv_orig);
        r->triple_counts = std::move(P->triple_counts);
        return;
    }
    // graph replay: the plan (buffers and instantiated graph) is kept on the
    // blocks handle per setting; replays of one plan are ordered on the
    // device through its `done` event
    std::lock_guard<std::mutex> lk(b->plan_mu);
    RunPlan* P = nullptr;
    for (auto& sp : b->run_plans) {
        RunPlan* q = static_cast<RunPlan*>(sp.get());
        if (q->same(o, o.variant, part_kind, core_k)) P = q;
    }
    if (!P) {
        std::unique_ptr<RunPlan> fresh = prepare(b, o, o.variant, part_kind, core_k, s);
        fresh->ctl.alloc(1, s);
        PGB_CUDA(cudaStreamSynchronize(s));  // plan inputs in place before capture
        capture(*fresh);
        if (b->run_plans.size() >= 4) b->run_plans.erase(b->run_plans.begin());
        P = fresh.get();
        b->run_plans.emplace_back(fresh.release(), [](void* q) { delete static_cast<RunPlan*>(q); });
    }
    if (P->used) PGB_CUDA(cudaStreamWaitEvent(s, P->done, 0));
    PGB_CUDA(cudaMemcpyAsync(P->ctl.ptr, &hctl, sizeof(RunCtl), cudaMemcpyHostToDevice, s));
    PGB_CUDA(cudaEventRecord(r->ev0, s));
    PGB_CUDA(cudaGraphLaunch(P->exec, s));
    note_launches(P->graph_launches);
    PGB_CUDA(cudaEventRecord(r->ev1, s));
    r->total.alloc(1, s);
    PGB_CUDA(cudaMemcpyAsync(r->total.ptr, P->total.ptr, 8, cudaMemcpyDeviceToDevice, s));
    keep_core_total(*P);
    PGB_CUDA(cudaMemcpyAsync(r->ctl.ptr, P->ctl.ptr, sizeof(RunCtl), cudaMemcpyDeviceToDevice, s));
    if (r->per_vertex) {
        r->tv_orig.alloc(n, s);
        if (n) PGB_CUDA(cudaMemcpyAsync(r->tv_orig.ptr, P->tv_orig.ptr, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
    }
    if (r->per_triple && r->ntriples) {
        r->triple_counts.alloc(r->ntriples, s);
        PGB_CUDA(cudaMemcpyAsync(r->triple_counts.ptr, P->triple_counts.ptr, r->ntriples * 8,
                                 cudaMemcpyDeviceToDevice, s));
    }
    PGB_CUDA(cudaEventRecord(P->done, s));
    P->used = true;
}

}  // namespace pgb

using namespace pgb;

extern "C" {

void pgb_tc_opts_default(pgb_tc_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->mode = PGB_MODE_PERSISTENT;
    o->variant = PGB_VAR_AUTO;
    o->per_vertex = 1;
    o->order = PGB_ORDER_WEIGHT;
}

int pgb_tc_run(const pgb_blocks* b, const pgb_tc_opts* opts, void* stream, pgb_tc_result** out) {
    return guard([&] {
        if (!b || !out) fail(PGB_E_INVAL, "NULL argument");
        pgb_tc_opts o;
        if (opts) o = *opts; else pgb_tc_opts_default(&o);
        if (o.mode != PGB_MODE_PLAIN && o.mode != PGB_MODE_PERSISTENT && o.mode != PGB_MODE_HYBRID)
            fail(PGB_E_INVAL, "bad mode");
        if (o.mode == PGB_MODE_HYBRID && (b->offloaded || o.use_graph))
            fail(PGB_E_STATE, "HYBRID runs need resident blocks and no graph replay");
        if (o.host_share_ppm > 1000000) fail(PGB_E_INVAL, "host_share_ppm must be at most 10^6");
        if (o.variant < PGB_VAR_AUTO || o.variant > PGB_VAR_HASH) fail(PGB_E_INVAL, "bad variant");
        if (o.mode == PGB_MODE_PLAIN && o.variant == PGB_VAR_HASH)
            fail(PGB_E_INVAL, "PLAIN mode runs the edge-wise variants (binary search, merge) only");
        if (o.order != PGB_ORDER_WEIGHT && o.order != PGB_ORDER_LOCALITY && o.order != PGB_ORDER_HILBERT)
            fail(PGB_E_INVAL, "bad order");
        if (o.hash_threads != 0 && o.hash_threads != 128 && o.hash_threads != 256 && o.hash_threads != 512)
            fail(PGB_E_INVAL, "hash_threads must be 0, 128, 256 or 512");
        if (b->offloaded && (o.mode != PGB_MODE_PERSISTENT || o.variant == PGB_VAR_BSEARCH ||
                             o.variant == PGB_VAR_MERGE))
            fail(PGB_E_STATE, "offloaded blocks run in PERSISTENT mode with the hash variant only");
        std::unique_ptr<pgb_tc_result> r(new pgb_tc_result());
        run(b, o, (cudaStream_t)stream, r.get());
        live_handles_add(1);
        *out = r.release();
    });
}

int pgb_tc_result_get(pgb_tc_result* r, uint64_t* total, uint64_t* per_vertex, int mem) {
    return guard([&] {
        if (!r) fail(PGB_E_INVAL, "result is NULL");
        cudaStream_t s = r->stream;
        uint32_t cancelled = 0;
        PGB_CUDA(cudaMemcpyAsync(&cancelled, &r->ctl.ptr->cancelled, 4, cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaStreamSynchronize(s));
        if (cancelled || r->host_cancelled)
            fail(PGB_E_CANCELLED, "the run stopped early on its cancel token; its counts are incomplete");
        if (per_vertex) {
            if (!r->per_vertex) fail(PGB_E_STATE, "run was made without per-vertex counts");
            copy_out(per_vertex, r->tv_orig.ptr, (size_t)r->n * 8, mem, s);
        }
        if (total) {
            unsigned long long h = 0;
            PGB_CUDA(cudaMemcpyAsync(&h, r->total.ptr, 8, cudaMemcpyDeviceToHost, s));
            PGB_CUDA(cudaStreamSynchronize(s));
            *total = h;
        }
        PGB_CUDA(cudaStreamSynchronize(s));
    });
}

int pgb_tc_result_triples(pgb_tc_result* r, uint64_t* counts, int mem) {
    return guard([&] {
        if (!r) fail(PGB_E_INVAL, "result is NULL");
        if (!r->per_triple) fail(PGB_E_STATE, "run was not PLAIN with per_triple = 1");
        copy_out(counts, r->triple_counts.ptr, r->ntriples * 8, mem, r->stream);
        PGB_CUDA(cudaStreamSynchronize(r->stream));
    });
}

int pgb_tc_result_variant(pgb_tc_result* r, int* variant) {
    return guard([&] {
        if (!r || !variant) fail(PGB_E_INVAL, "NULL argument");
        *variant = r->variant;
    });
}

int pgb_tc_result_dense_core(pgb_tc_result* r, pgb_dense_core_info* out) {
    return guard([&] {
        if (!r || !out) fail(PGB_E_INVAL, "NULL argument");
        std::memset(out, 0, sizeof(*out));
        out->ms = -1.0f;
        out->ranks = r->core_ranks;
        if (!r->core_ranks) return;
        unsigned long long t = 0;
        PGB_CUDA(cudaMemcpyAsync(&t, r->core_total.ptr, 8, cudaMemcpyDeviceToHost, r->stream));
        PGB_CUDA(cudaStreamSynchronize(r->stream));
        out->triangles = t;
        out->lookups_skipped = r->core_lookups;
        out->gemm_flop = r->core_flop;
        if (r->evc0 && r->evc1) PGB_CUDA(cudaEventElapsedTime(&out->ms, r->evc0, r->evc1));
    });
}

int pgb_tc_result_part_variants(pgb_tc_result* r, uint32_t* p, int32_t* variants) {
    return guard([&] {
        if (!r || !p) fail(PGB_E_INVAL, "NULL argument");
        *p = (uint32_t)r->part_variant.size();
        if (variants && !r->part_variant.empty())
            std::memcpy(variants, r->part_variant.data(), r->part_variant.size() * sizeof(int32_t));
    });
}

int pgb_tc_result_hybrid(pgb_tc_result* r, float* host_ms, uint64_t* host_in_edges, uint32_t* host_parts,
                         uint32_t* host_threads) {
    return guard([&] {
        if (!r) fail(PGB_E_INVAL, "result is NULL");
        if (host_ms) *host_ms = r->host_ms;
        if (host_in_edges) *host_in_edges = r->host_in_edges;
        if (host_parts) *host_parts = r->host_parts;
        if (host_threads) *host_threads = r->host_threads;
    });
}

int pgb_tc_result_stream(pgb_tc_result* r, uint64_t* bytes, uint32_t* chunks, uint32_t* slice_loads) {
    return guard([&] {
        if (!r || !bytes || !chunks) fail(PGB_E_INVAL, "NULL argument");
        *bytes = r->streamed;
        *chunks = r->chunks;
        if (slice_loads) *slice_loads = r->slice_loads;
    });
}

int pgb_tc_result_kernel_ms(pgb_tc_result* r, float* ms) {
    return guard([&] {
        if (!r || !ms) fail(PGB_E_INVAL, "NULL argument");
        PGB_CUDA(cudaEventSynchronize(r->ev1));
        PGB_CUDA(cudaEventElapsedTime(ms, r->ev0, r->ev1));
    });
}

void pgb_tc_result_free(pgb_tc_result* r) {
    if (!r) return;
    delete r;
    live_handles_add(-1);
}

int pgb_tc_count_edges(const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n, uint32_t p,
                       int cut_rule, const pgb_tc_opts* opts, int mem, void* stream, uint64_t* total,
                       uint64_t* per_vertex) {
    pgb_graph* g = nullptr;
    pgb_blocks* b = nullptr;
    pgb_tc_result* r = nullptr;
    int rc = pgb_graph_from_edges(src, dst, m, n, mem, stream, &g);
    if (rc == PGB_OK) rc = pgb_partition(g, p, cut_rule, stream, &b);
    pgb_graph_free(g);
    pgb_tc_opts o;
    if (opts) o = *opts; else pgb_tc_opts_default(&o);
    if (!per_vertex) o.per_vertex = 0;
    if (rc == PGB_OK) rc = pgb_tc_run(b, &o, stream, &r);
    if (rc == PGB_OK) rc = pgb_tc_result_get(r, total, per_vertex, mem);
    pgb_tc_result_free(r);
    pgb_blocks_free(b);
    return rc;
}

}  // extern "C"
