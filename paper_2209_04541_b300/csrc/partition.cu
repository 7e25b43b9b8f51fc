// Degree ordering, upper orientation, p x p partition and block-triple
// queue (Sections 3.6, 4.3, 4.4 and 5.4 of PGAbB).
//
// Layout produced (all on the device, rank space):
//   perm[r]     original ID of rank r (ranks sort vertices by (degree, ID))
//   rowptr/col  oriented CSR: row u lists v > u ascending (uint32 offsets;
//               the library rejects graphs with 2^32 or more edges)
//   rowidx[e]   row of oriented edge e
//   bedge       edge positions grouped by block (i, j) in row-major block
//               order (Section 4.3 "row-major order"), CSR order inside a
//               block; block (i, j) occupies [block_off[ij], block_off[ij+1])
// Because every part is a contiguous rank range, the partial list of u in
// block A_ik is the contiguous slice of row u with columns in [c_k, c_k+1).

#include <algorithm>
#include <memory>
#include <mutex>
#include <numeric>

#include "core.cuh"
#include "internal.cuh"
#include "sort.cuh"

namespace pgb {

static int grid_for(uint64_t items, int threads = 256) {
    uint64_t g = (items + threads - 1) / threads;
    if (g > 148ull * 32) g = 148ull * 32;
    return g < 1 ? 1 : (int)g;
}

__global__ void k_iota(uint32_t* __restrict__ x, uint64_t n) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) x[i] = (uint32_t)i;
}

__global__ void k_invert(const uint32_t* __restrict__ perm, uint32_t n, uint32_t* __restrict__ rank) {
    uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) rank[perm[r]] = r;
}

// Oriented endpoints of each undirected edge: its lower rank (the row) and
// its higher rank (the column).
__global__ void k_orient_pairs(const uint64_t* __restrict__ keys, uint64_t m, uint32_t B,
                               const uint32_t* __restrict__ rank, uint32_t* __restrict__ row,
                               uint32_t* __restrict__ colv) {
    const uint64_t mask = (1ull << B) - 1;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        uint64_t k = keys[e];
        uint32_t ra = rank[(uint32_t)(k >> B)], rb = rank[(uint32_t)(k & mask)];
        row[e] = ra < rb ? ra : rb;
        colv[e] = ra < rb ? rb : ra;
    }
}

// Offsets of a sorted key array: off[r] = first position whose key is >= r,
// for r in [0, n] (one binary search per entry, so runs of empty rows cost
// nothing extra).
__global__ void k_offsets_from_sorted(const uint32_t* __restrict__ keys, uint64_t m, uint32_t n,
                                      uint32_t* __restrict__ off) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= n; r += stride) {
        uint64_t lo = 0, hi = m;
        while (lo < hi) {
            uint64_t mid = (lo + hi) >> 1;
            if (keys[mid] < r) lo = mid + 1; else hi = mid;
        }
        off[r] = (uint32_t)lo;
    }
}

// Tail-row range of every edge: for the edge u -> v at CSR position e, the
// entries of u's row after v, packed as (e + 1) | (rowptr[u + 1] << 32), with
// its head v as the sort key; both are written in reverse CSR order, so that
// the stable sort on the head leaves each head's tails descending (measured
// 5% faster counting at R-MAT scale 24 than ascending).  Also sums the range
// lengths (the lookups of the middle-vertex variant).
__global__ void k_row_ranges(uint64_t m, const uint32_t* __restrict__ rowidx, const uint32_t* __restrict__ rowptr,
                             unsigned long long* __restrict__ xa, unsigned long long* __restrict__ probes,
                             const uint32_t* __restrict__ col, uint32_t* __restrict__ kout) {
    unsigned long long acc = 0;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const uint32_t xe = rowptr[rowidx[e] + 1];
        xa[m - 1 - e] = (unsigned long long)(e + 1) | ((unsigned long long)xe << 32);
        kout[m - 1 - e] = col[e];
        acc += xe - (uint32_t)(e + 1);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(probes, acc);
}

__global__ void k_fill_u32(uint32_t* __restrict__ x, uint64_t n, uint32_t v) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) x[i] = v;
}

// Cut points.  NNZ rule: c[t] = least r in [0, n] with rowptr[r] * p >= t * M,
// found by binary search over the non-decreasing rowptr.  UNIFORM rule:
// c[t] = floor(t * n / p).
__global__ void k_cuts(const uint32_t* __restrict__ rowptr, uint32_t n, uint32_t p, int rule,
                       uint32_t* __restrict__ cuts) {
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > p) return;
    if (t == 0) { cuts[0] = 0; return; }
    if (t == p) { cuts[p] = n; return; }
    if (rule == PGB_CUT_UNIFORM) {
        cuts[t] = (uint32_t)(((uint64_t)t * n) / p);
        return;
    }
    const uint64_t M = rowptr[n];
    const uint64_t need = (uint64_t)t * M;
    uint32_t lo = 0, hi = n + 1;  // first r in [0, n] with rowptr[r] * p >= need
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if ((uint64_t)rowptr[mid] * p >= need) hi = mid; else lo = mid + 1;
    }
    cuts[t] = lo;
}

__device__ __forceinline__ uint32_t part_of(const uint32_t* cuts, uint32_t p, uint32_t r) {
    // largest t in [0, p) with cuts[t] <= r
    uint32_t lo = 0, hi = p;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (cuts[mid] <= r) lo = mid; else hi = mid;
    }
    return lo;
}

// Block id (i * p + j) of every oriented edge (when bid is not null) and the
// p x p block edge histogram (when hist is not null; shared-memory counters
// when p*p fits, global otherwise).  With part_probes not null, also the
// lookups of the middle-vertex variant per head part j: the sum over edges
// (u, v) with v in V_j of the entries of u's row after v (shared counters).
__global__ void k_block_ids(const uint32_t* __restrict__ rowidx, const uint32_t* __restrict__ col, uint64_t m,
                            const uint32_t* __restrict__ cuts_g, uint32_t p, uint32_t* __restrict__ bid,
                            unsigned long long* __restrict__ hist, const uint32_t* __restrict__ rowptr,
                            unsigned long long* __restrict__ part_probes) {
    extern __shared__ unsigned long long sm64[];
    unsigned long long* pp_s = sm64;  // p entries when part_probes is set
    uint32_t* cuts = reinterpret_cast<uint32_t*>(sm64 + (part_probes ? p : 0));
    uint32_t* h = cuts + p + 1;
    const bool use_smem = (uint64_t)p * p <= 4096;
    for (uint32_t i = threadIdx.x; i <= p; i += blockDim.x) cuts[i] = cuts_g[i];
    if (use_smem)
        for (uint32_t i = threadIdx.x; i < p * p; i += blockDim.x) h[i] = 0;
    if (part_probes)
        for (uint32_t i = threadIdx.x; i < p; i += blockDim.x) pp_s[i] = 0;
    __syncthreads();
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e0 = (uint64_t)blockIdx.x * blockDim.x; e0 < m; e0 += stride) {
        const uint64_t e = e0 + threadIdx.x;
        const bool live = e < m;
        uint32_t j = 0xffffffffu, after = 0;
        if (live) {
            const uint32_t u = rowidx[e];
            j = part_of(cuts, p, col[e]);
            const uint32_t b = part_of(cuts, p, u) * p + j;
            if (bid) bid[e] = b;
            if (part_probes) after = rowptr[u + 1] - (uint32_t)(e + 1);
            if (hist) {
                if (use_smem) atomicAdd(&h[b], 1u);
                else atomicAdd(&hist[b], 1ull);
            }
        }
        if (part_probes) {
            // a warp's edges are consecutive CSR positions, so their heads
            // fall into few parts: one shared atomic per part and warp
            const unsigned act = __ballot_sync(0xffffffffu, live);
            if (live) {
                const unsigned grp = __match_any_sync(act, j);
                const uint32_t sum = __reduce_add_sync(grp, after);
                // (32 of them stay below 2^32: with degree order an out-degree
            // is at most sqrt(2 m) < 92,700 for m < 2^32)
            if ((threadIdx.x & 31) == (unsigned)(__ffs(grp) - 1) && sum)
                    atomicAdd(&pp_s[j], (unsigned long long)sum);
            }
        }
    }
    if ((use_smem && hist) || part_probes) __syncthreads();
    if (use_smem && hist) {
        for (uint32_t i = threadIdx.x; i < p * p; i += blockDim.x)
            if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
    }
    if (part_probes)
        for (uint32_t i = threadIdx.x; i < p; i += blockDim.x)
            if (pp_s[i]) atomicAdd(&part_probes[i], pp_s[i]);
}

// out[t] = colptr[cuts[t]] for t <= p: where each head part's in-edges start.
__global__ void k_head_offsets(const uint32_t* __restrict__ colptr, const uint32_t* __restrict__ cuts, uint32_t p,
                               unsigned long long* __restrict__ out) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t <= p) out[t] = colptr[cuts[t]];
}

// sum_v indeg(v) * outdeg(v) and max outdeg.
__global__ void k_wedges(const uint32_t* __restrict__ colptr, const uint32_t* __restrict__ rowptr, uint32_t n,
                         unsigned long long* __restrict__ out_sum, unsigned int* __restrict__ out_max) {
    __shared__ unsigned long long ssum[32];
    __shared__ unsigned int smax[32];
    unsigned long long acc = 0;
    unsigned int mx = 0;
    uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        uint32_t od = rowptr[v + 1] - rowptr[v];
        acc += (unsigned long long)(colptr[v + 1] - colptr[v]) * od;
        mx = od > mx ? od : mx;
    }
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_down_sync(0xffffffffu, acc, o);
        unsigned int y = __shfl_down_sync(0xffffffffu, mx, o);
        mx = y > mx ? y : mx;
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { ssum[w] = acc; smax[w] = mx; }
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        acc = l < nw ? ssum[l] : 0;
        mx = l < nw ? smax[l] : 0;
        for (int o = 16; o > 0; o >>= 1) {
            acc += __shfl_down_sync(0xffffffffu, acc, o);
            unsigned int y = __shfl_down_sync(0xffffffffu, mx, o);
            mx = y > mx ? y : mx;
        }
        if (l == 0) {
            atomicAdd(out_sum, acc);
            atomicMax(out_max, mx);
        }
    }
}

// Section 3.6 block-list composition with the Section 4.4 default weight
// (edges in the block-list) and decreasing order; ties by (i, j, k).
static std::vector<pgb_triple> make_queue(uint32_t p, const std::vector<uint64_t>& be) {
    std::vector<pgb_triple> q;
    for (uint32_t i = 0; i < p; ++i)
        for (uint32_t j = i; j < p; ++j) {
            uint64_t a = be[(size_t)i * p + j];
            if (!a) continue;
            for (uint32_t k = j; k < p; ++k) {
                uint64_t b = be[(size_t)i * p + k], c = be[(size_t)j * p + k];
                if (b && c) q.push_back({i, j, k, a + b + c});
            }
        }
    std::stable_sort(q.begin(), q.end(), [](const pgb_triple& x, const pgb_triple& y) { return x.w > y.w; });
    return q;
}

void build_partition(const pgb_graph* g, uint32_t p, int rule, cudaStream_t s, pgb_blocks* b) {
    const uint32_t n = g->n;
    const uint64_t m = g->m;
    const uint32_t B = g->id_bits;
    b->n = n;
    b->p = p;
    b->m = m;
    b->stream = s;
    Scratch scratch;

    // --- degree order: stable sort of IDs by degree (ties keep ID order)
    b->perm.alloc(n, s);
    DevBuf<uint32_t> rank(n, s);
    if (n > 0) {
        DevBuf<uint32_t> kd(n, s), kalt(n, s), ids(n, s);
        PGB_CUDA(cudaMemcpyAsync(kd.ptr, g->deg.ptr, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
        k_iota<<<grid_for(n), 256, 0, s>>>(ids.ptr, n);
        PGB_CHECK_LAUNCH("k_iota");
        uint32_t *ko, *vo;
        sort_pairs(kd.ptr, kalt.ptr, ids.ptr, b->perm.ptr, n, num_bits(n), s, scratch, &ko, &vo);
        if (vo != b->perm.ptr)
            PGB_CUDA(cudaMemcpyAsync(b->perm.ptr, vo, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
        k_invert<<<grid_for(n), 256, 0, s>>>(b->perm.ptr, n, rank.ptr);
        PGB_CHECK_LAUNCH("k_invert");
    }

    // --- orientation: sort (low rank, high rank) pairs
    b->rowptr.alloc((size_t)n + 1, s);
    // 8 spare entries: the counting kernels read rows with aligned 32-byte
    // loads, whose last load may extend up to 7 entries past the last edge
    b->col.alloc(m + 8, s);
    PGB_CUDA(cudaMemsetAsync(b->col.ptr + m, 0, 32, s));
    b->rowidx.alloc(m, s);
    if (m > 0) {
        // rows and columns are sorted in two extra arrays plus rowidx and
        // col themselves; the result is copied over when it lands in the
        // extra pair
        DevBuf<uint32_t> ra(m, s), ca(m, s);
        k_orient_pairs<<<grid_for(m), 256, 0, s>>>(g->keys.ptr, m, B, rank.ptr, ra.ptr, ca.ptr);
        PGB_CHECK_LAUNCH("k_orient_pairs");
        uint32_t *ro, *co;
        sort_pairs_lex(ra.ptr, b->rowidx.ptr, ca.ptr, b->col.ptr, m, (int)B, s, scratch, &ro, &co);
        if (ro != b->rowidx.ptr) PGB_CUDA(cudaMemcpyAsync(b->rowidx.ptr, ro, m * 4, cudaMemcpyDeviceToDevice, s));
        if (co != b->col.ptr) PGB_CUDA(cudaMemcpyAsync(b->col.ptr, co, m * 4, cudaMemcpyDeviceToDevice, s));
        k_offsets_from_sorted<<<grid_for((uint64_t)n + 1), 256, 0, s>>>(b->rowidx.ptr, m, n, b->rowptr.ptr);
        PGB_CHECK_LAUNCH("k_offsets_from_sorted");
    } else {
        k_fill_u32<<<grid_for((uint64_t)n + 1), 256, 0, s>>>(b->rowptr.ptr, (uint64_t)n + 1, 0);
        PGB_CHECK_LAUNCH("k_fill_u32");
    }
    rank.release();

    // --- cuts
    b->cuts_d.alloc((size_t)p + 1, s);
    k_cuts<<<(p + 1 + 127) / 128, 128, 0, s>>>(b->rowptr.ptr, n, p, rule, b->cuts_d.ptr);
    PGB_CHECK_LAUNCH("k_cuts");
    b->cuts.assign((size_t)p + 1, 0);

    // --- block histogram (per-edge block ids are built on demand, for the
    // runs that walk edges block by block)
    const size_t pp = (size_t)p * p;
    // p x p histogram, the per-part lookups (p), the head parts' in-edge
    // offsets (p + 1), the lookups per top-rank band (kCoreBands)
    const size_t nhist = pp + 2 * (size_t)p + 1 + kCoreBands;
    DevBuf<unsigned long long> hist(nhist, s);
    PGB_CUDA(cudaMemsetAsync(hist.ptr, 0, nhist * 8, s));
    if (m > 0) {
        size_t smem = (size_t)p * 8 + ((size_t)p + 1) * 4 + (pp <= 4096 ? pp * 4 : 0);
        k_block_ids<<<grid_for(m), 256, smem, s>>>(b->rowidx.ptr, b->col.ptr, m, b->cuts_d.ptr, p, nullptr,
                                                   hist.ptr, b->rowptr.ptr, hist.ptr + pp);
        PGB_CHECK_LAUNCH("k_block_ids");
    }

    // --- in-edge index for the middle-vertex variant: each edge's tail-row
    // range after its head, made in reverse CSR order, then carried into head
    // order by a stable radix sort on the head (tails descend within a head);
    // colptr[v] = first in-edge of v.  Wedge statistics use in-degrees
    // colptr[v + 1] - colptr[v].
    b->colptr.alloc((size_t)n + 1, s);
    b->xr.alloc(m, s);
    DevBuf<unsigned long long> wsum(1, s), wprobe(1, s);
    DevBuf<unsigned int> wmax(1, s);
    PGB_CUDA(cudaMemsetAsync(wsum.ptr, 0, 8, s));
    PGB_CUDA(cudaMemsetAsync(wprobe.ptr, 0, 8, s));
    PGB_CUDA(cudaMemsetAsync(wmax.ptr, 0, 4, s));
    if (m > 0) {
        DevBuf<uint32_t> kc(m, s), kalt(m, s);
        DevBuf<unsigned long long> xa(m, s);
        k_row_ranges<<<grid_for(m), 256, 0, s>>>(m, b->rowidx.ptr, b->rowptr.ptr, xa.ptr, wprobe.ptr, b->col.ptr, kc.ptr);
        PGB_CHECK_LAUNCH("k_row_ranges");
        uint32_t* ko;
        unsigned long long* vo;
        sort_pairs(kc.ptr, kalt.ptr, xa.ptr, b->xr.ptr, m, num_bits(n > 0 ? n - 1 : 0), s, scratch, &ko, &vo);
        if (vo != b->xr.ptr) PGB_CUDA(cudaMemcpyAsync(b->xr.ptr, vo, m * 8, cudaMemcpyDeviceToDevice, s));
        k_offsets_from_sorted<<<grid_for((uint64_t)n + 1), 256, 0, s>>>(ko, m, n, b->colptr.ptr);
        PGB_CHECK_LAUNCH("k_offsets_from_sorted");
        k_wedges<<<grid_for(n), 256, 0, s>>>(b->colptr.ptr, b->rowptr.ptr, n, wsum.ptr, wmax.ptr);
        PGB_CHECK_LAUNCH("k_wedges");
        k_head_offsets<<<(p + 1 + 127) / 128, 128, 0, s>>>(b->colptr.ptr, b->cuts_d.ptr, p, hist.ptr + pp + p);
        PGB_CHECK_LAUNCH("k_head_offsets");
    } else {
        k_fill_u32<<<grid_for((uint64_t)n + 1), 256, 0, s>>>(b->colptr.ptr, (uint64_t)n + 1, 0);
        PGB_CHECK_LAUNCH("k_fill_u32");
    }

    core_band_probes(b, hist.ptr + pp + 2 * (size_t)p + 1, s);

    // --- one sync: cuts, histogram, stats to the host
    b->block_edges.assign(pp, 0);
    b->part_probes.assign(p, 0);
    unsigned long long hw = 0, hp = 0;
    unsigned int hm = 0;
    PGB_CUDA(cudaMemcpyAsync(b->cuts.data(), b->cuts_d.ptr, ((size_t)p + 1) * 4, cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaMemcpyAsync(b->block_edges.data(), hist.ptr, pp * 8, cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaMemcpyAsync(b->part_probes.data(), hist.ptr + pp, (size_t)p * 8, cudaMemcpyDeviceToHost, s));
    b->head_off.assign((size_t)p + 1, 0);
    PGB_CUDA(cudaMemcpyAsync(b->head_off.data(), hist.ptr + pp + p, ((size_t)p + 1) * 8, cudaMemcpyDeviceToHost, s));
    b->core_probes.assign(kCoreBands, 0);
    PGB_CUDA(cudaMemcpyAsync(b->core_probes.data(), hist.ptr + pp + 2 * (size_t)p + 1, kCoreBands * 8,
                             cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaMemcpyAsync(&hw, wsum.ptr, 8, cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaMemcpyAsync(&hp, wprobe.ptr, 8, cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaMemcpyAsync(&hm, wmax.ptr, 4, cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaStreamSynchronize(s));
    b->wedges = hw;
    b->probes = hp;
    b->max_outdeg = hm;
    b->block_off.assign(pp + 1, 0);
    for (size_t i = 0; i < pp; ++i) b->block_off[i + 1] = b->block_off[i] + b->block_edges[i];
    b->triples = make_queue(p, b->block_edges);
}

// Block-grouped edge index (positions of the edges of block (i, j), blocks in
// row-major order, CSR order inside a block): a stable radix sort of
// (block id, edge position).  Built once per partition, on first use.
void ensure_block_edge_index(const pgb_blocks* b, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(b->bedge_mu);
    if (b->bedge_ready) return;
    const uint64_t m = b->m;
    const uint32_t p = b->p;
    b->bedge.alloc(m, s);
    if (m > 0) {
        if (p == 1) {
            k_iota<<<grid_for(m), 256, 0, s>>>(b->bedge.ptr, m);
            PGB_CHECK_LAUNCH("k_iota");
        } else {
            Scratch scratch;
            const size_t pp = (size_t)p * p;
            DevBuf<uint32_t> bid(m, s), kalt(m, s), vals(m, s);
            size_t smem = ((size_t)p + 1) * 4 + (pp <= 4096 ? pp * 4 : 0);
            k_block_ids<<<grid_for(m), 256, smem, s>>>(b->rowidx.ptr, b->col.ptr, m, b->cuts_d.ptr, p, bid.ptr,
                                                       nullptr, nullptr, nullptr);
            PGB_CHECK_LAUNCH("k_block_ids");
            k_iota<<<grid_for(m), 256, 0, s>>>(vals.ptr, m);
            PGB_CHECK_LAUNCH("k_iota");
            uint32_t *ko, *vo;
            sort_pairs(bid.ptr, kalt.ptr, vals.ptr, b->bedge.ptr, m, num_bits(pp - 1), s, scratch, &ko, &vo);
            if (vo != b->bedge.ptr)
                PGB_CUDA(cudaMemcpyAsync(b->bedge.ptr, vo, m * 4, cudaMemcpyDeviceToDevice, s));
        }
    }
    b->bedge_ready = true;
}

}  // namespace pgb

using namespace pgb;

extern "C" {

int pgb_partition(const pgb_graph* g, uint32_t p, int cut_rule, void* stream, pgb_blocks** out) {
    return guard([&] {
        if (!g || !out) fail(PGB_E_INVAL, "NULL argument");
        if (p == 0 || p > 1024) fail(PGB_E_INVAL, "p must be in [1, 1024]");
        if (g->n > 0 && p > g->n) fail(PGB_E_INVAL, "p must not exceed n");
        if (cut_rule != PGB_CUT_NNZ && cut_rule != PGB_CUT_UNIFORM) fail(PGB_E_INVAL, "bad cut rule");
        if (g->n == 0xFFFFFFFFu) fail(PGB_E_OVERFLOW, "n must be below 2^32 - 1");
        std::unique_ptr<pgb_blocks> b(new pgb_blocks());
        build_partition(g, p, cut_rule, (cudaStream_t)stream, b.get());
        live_handles_add(1);
        *out = b.release();
    });
}

int pgb_blocks_info(const pgb_blocks* b, pgb_blocks_stats* out) {
    return guard([&] {
        if (!b || !out) fail(PGB_E_INVAL, "NULL argument");
        std::memset(out, 0, sizeof(*out));
        out->n = b->n;
        out->p = b->p;
        out->m = b->m;
        uint64_t ne = 0;
        for (uint64_t x : b->block_edges) ne += x ? 1 : 0;
        out->nonempty_blocks = ne;
        out->triples = b->triples.size();
        out->wedges = b->wedges;
        out->alg_bytes = 4 * b->m + 4 * b->wedges + 8 * ((uint64_t)b->n + 1);
        out->max_outdeg = b->max_outdeg;
        out->probes = b->probes;
    });
}

__global__ void k_widen(const uint32_t* __restrict__ x, uint64_t n, int64_t* __restrict__ y) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) y[i] = x[i];
}

int pgb_blocks_export(const pgb_blocks* b, int what, void* dst, int mem, void* stream) {
    return guard([&] {
        if (!b) fail(PGB_E_INVAL, "blocks is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        auto host_or_dev = [&](const void* hsrc, size_t bytes) {
            if (!bytes) return;
            if (!dst) fail(PGB_E_INVAL, "NULL destination");
            if (mem == PGB_MEM_DEVICE) {
                PGB_CUDA(cudaMemcpyAsync(dst, hsrc, bytes, cudaMemcpyHostToDevice, s));
                PGB_CUDA(cudaStreamSynchronize(s));
            } else {
                std::memcpy(dst, hsrc, bytes);
            }
        };
        switch (what) {
            case PGB_EXPORT_PERM: copy_out(dst, b->perm.ptr, (size_t)b->n * 4, mem, s); break;
            case PGB_EXPORT_ROWPTR: {
                DevBuf<int64_t> w((size_t)b->n + 1, s);
                k_widen<<<grid_for((uint64_t)b->n + 1), 256, 0, s>>>(b->rowptr.ptr, (uint64_t)b->n + 1, w.ptr);
                PGB_CHECK_LAUNCH("k_widen");
                copy_out(dst, w.ptr, ((size_t)b->n + 1) * 8, mem, s);
                PGB_CUDA(cudaStreamSynchronize(s));
                break;
            }
            case PGB_EXPORT_COL:
                if (b->cols_offloaded) {
                    if (b->m)
                        PGB_CUDA(cudaMemcpyAsync(dst, offloaded_columns(b), b->m * 4, cudaMemcpyDefault, s));
                } else {
                    copy_out(dst, b->col.ptr, b->m * 4, mem, s);
                }
                break;
            case PGB_EXPORT_CUTS: host_or_dev(b->cuts.data(), b->cuts.size() * 4); break;
            case PGB_EXPORT_BLOCK_EDGES: host_or_dev(b->block_edges.data(), b->block_edges.size() * 8); break;
            case PGB_EXPORT_PART_PROBES: host_or_dev(b->part_probes.data(), b->part_probes.size() * 8); break;
            case PGB_EXPORT_TRIPLES: {
                std::vector<uint32_t> t(3 * b->triples.size());
                for (size_t i = 0; i < b->triples.size(); ++i) {
                    t[3 * i] = b->triples[i].i;
                    t[3 * i + 1] = b->triples[i].j;
                    t[3 * i + 2] = b->triples[i].k;
                }
                host_or_dev(t.data(), t.size() * 4);
                break;
            }
            case PGB_EXPORT_WEIGHTS: {
                std::vector<uint64_t> w(b->triples.size());
                for (size_t i = 0; i < w.size(); ++i) w[i] = b->triples[i].w;
                host_or_dev(w.data(), w.size() * 8);
                break;
            }
            default: fail(PGB_E_INVAL, "unknown export id");
        }
    });
}

void pgb_blocks_free(pgb_blocks* b) {
    if (!b) return;
    delete b;
    live_handles_add(-1);
}

}  // extern "C"
