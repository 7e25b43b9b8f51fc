// Other multi-block pattern counts on the block store (PGAbB Section 3.2:
// k-clique finding and butterfly counting compose block-lists of several
// blocks, like triangle counting): 4-cliques and 4-cycles.
//
// Both run in rank space on the degree-ordered oriented graph.
//
// 4-cliques.  A 4-clique u < v < w < x is found once, from its lowest edge
// (u, v): w is a common out-neighbour of u and v, and x a common
// out-neighbour of u, v and w above w.  The block-list of the clique is the
// six blocks of its vertex pairs; the kernel visits every oriented edge, so
// every block-list's work is covered.  One warp per edge: the lanes take the
// candidates w of u's row after v and binary-search each in v's row; for a
// hit, the lane walks the shortest of the three lists that x must lie in
// (u's row after w, v's row after w, w's row) and binary-searches the
// other two.
//
// 4-cycles.  Vertex priority by rank: a 4-cycle is counted once, at its
// highest-ranked vertex a, with b the vertex opposite a and w, y its two
// neighbours on the cycle (all ranked below a).  For each a, every path
// a - w - b with w, b < a adds 1 to a counter of b; a pair {a, b} with c such
// paths closes C(c, 2) cycles, summed without a second pass by adding the
// counter's old value at each increment (0 + 1 + ... + (c - 1)).  A second
// walk over the same paths clears the counters.  Each CTA owns a dense
// counter array of n words in device memory; the number of CTAs is bounded
// by a memory budget.  Lower neighbours of a vertex are its in-edge tails;
// its upper neighbours below a are the prefix of its row up to a.  On a
// bipartite graph the 4-cycles are its butterflies.
#include <algorithm>

#include "internal.cuh"

namespace pgb {

namespace {

constexpr int kPatThreads = 256;
constexpr int kPatWarps = kPatThreads / 32;
constexpr int kC4Threads = 512;
constexpr uint64_t kC4CounterBudget = 8ull << 30;  // bytes of per-CTA counter arrays

__device__ __forceinline__ uint32_t lb(const uint32_t* __restrict__ a, uint32_t b, uint32_t e, uint32_t x) {
    uint32_t n = e - b;
    while (n > 0) {
        const uint32_t half = n >> 1;
        if (__ldg(a + b + half) < x) {
            b += half + 1;
            n -= half + 1;
        } else {
            n = half;
        }
    }
    return b;
}

__device__ __forceinline__ bool has(const uint32_t* __restrict__ a, uint32_t b, uint32_t e, uint32_t x) {
    const uint32_t p = lb(a, b, e, x);
    return p < e && __ldg(a + p) == x;
}

__device__ __forceinline__ void cta_total(unsigned long long cnt, unsigned long long* __restrict__ slot, int warps) {
    __shared__ unsigned long long red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if (lane == 0) red[warp] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < warps; ++w) t += red[w];
        *slot = t;
    }
}

__global__ void __launch_bounds__(kPatThreads)
    k_k4(const uint32_t* __restrict__ rowptr, const uint32_t* __restrict__ rowidx, const uint32_t* __restrict__ col,
         uint32_t m, unsigned long long* __restrict__ partials) {
    const int lane = threadIdx.x & 31;
    const uint32_t gw = blockIdx.x * kPatWarps + (threadIdx.x >> 5), nw = gridDim.x * kPatWarps;
    unsigned long long cnt = 0;
    for (uint32_t e = gw; e < m; e += nw) {
        const uint32_t u = __ldg(rowidx + e), v = __ldg(col + e);
        const uint32_t ue = __ldg(rowptr + u + 1);
        const uint32_t vb = __ldg(rowptr + v), ve = __ldg(rowptr + v + 1);
        if (vb == ve) continue;
        for (uint32_t i = e + 1 + lane; i < ue; i += 32) {
            const uint32_t w = __ldg(col + i);
            const uint32_t pv = lb(col, vb, ve, w);
            if (pv >= ve || __ldg(col + pv) != w) continue;
            // x lies in u's row after w [i+1, ue), v's row after w [pv+1, ve)
            // and w's row: walk the shortest, search the other two
            const uint32_t wb = __ldg(rowptr + w), we = __ldg(rowptr + w + 1);
            uint32_t ab = i + 1, ae = ue, bb = pv + 1, be = ve, cb = wb, ce = we;
            if (be - bb < ae - ab) {
                uint32_t t0 = ab, t1 = ae;
                ab = bb; ae = be; bb = t0; be = t1;
            }
            if (ce - cb < ae - ab) {
                uint32_t t0 = ab, t1 = ae;
                ab = cb; ae = ce; cb = t0; ce = t1;
            }
            for (uint32_t k = ab; k < ae; ++k) {
                const uint32_t x = __ldg(col + k);
                if (has(col, bb, be, x) && has(col, cb, ce, x)) ++cnt;
            }
        }
    }
    cta_total(cnt, partials + blockIdx.x, kPatWarps);
}

// The paths a - w - b with w, b < a: w over a's in-edge tails (one warp per
// tail), b over w's in-edge tails and the part of w's row below a.  Pass 0
// counts (adding each counter's old value), pass 1 clears.
template <int kPass>
__device__ __forceinline__ unsigned long long c4_paths(uint32_t a, const uint32_t* __restrict__ rowptr,
                                                       const uint32_t* __restrict__ col,
                                                       const uint32_t* __restrict__ colptr,
                                                       const uint32_t* __restrict__ itail, uint32_t* __restrict__ cnt) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kWarps = kC4Threads / 32;
    unsigned long long acc = 0;
    const uint32_t qb = __ldg(colptr + a), qe = __ldg(colptr + a + 1);
    for (uint32_t q = qb + warp; q < qe; q += kWarps) {
        const uint32_t w = __ldg(itail + q);
        const uint32_t tb = __ldg(colptr + w), te = __ldg(colptr + w + 1);
        for (uint32_t t = tb + lane; t < te; t += 32) {
            const uint32_t b = __ldg(itail + t);
            if (kPass == 0) acc += atomicAdd(cnt + b, 1u);
            else cnt[b] = 0;
        }
        const uint32_t rb = __ldg(rowptr + w);
        const uint32_t re = lb(col, rb, __ldg(rowptr + w + 1), a);  // row entries below a
        for (uint32_t r = rb + lane; r < re; r += 32) {
            const uint32_t b = __ldg(col + r);
            if (kPass == 0) acc += atomicAdd(cnt + b, 1u);
            else cnt[b] = 0;
        }
    }
    return acc;
}

__global__ void __launch_bounds__(kC4Threads)
    k_c4(const uint32_t* __restrict__ rowptr, const uint32_t* __restrict__ col, const uint32_t* __restrict__ colptr,
         const uint32_t* __restrict__ itail, uint32_t n, uint32_t* __restrict__ counters, uint64_t stride_words,
         unsigned int* __restrict__ cursor, unsigned long long* __restrict__ partials) {
    __shared__ uint32_t s_a;
    uint32_t* cnt = counters + (uint64_t)blockIdx.x * stride_words;
    unsigned long long acc = 0;
    for (;;) {
        if (threadIdx.x == 0) s_a = atomicAdd(cursor, 1u);
        __syncthreads();
        const uint32_t k = s_a;
        __syncthreads();
        if (k >= n) break;
        const uint32_t a = n - 1 - k;  // top ranks (most paths) first
        acc += c4_paths<0>(a, rowptr, col, colptr, itail, cnt);
        __syncthreads();
        c4_paths<1>(a, rowptr, col, colptr, itail, cnt);
        __syncthreads();
    }
    cta_total(acc, partials + blockIdx.x, kC4Threads / 32);
}

__global__ void k_sum_u64(const unsigned long long* __restrict__ p, uint32_t k, unsigned long long* __restrict__ out) {
    __shared__ unsigned long long red[32];
    unsigned long long s = 0;
    for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) s += p[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (uint32_t w = 0; w < (blockDim.x >> 5); ++w) t += red[w];
        *out = t;
    }
}

__global__ void k_tails_of(const unsigned long long* __restrict__ xr, const uint32_t* __restrict__ rowidx, uint64_t m,
                           uint32_t* __restrict__ itail) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += stride)
        itail[q] = rowidx[(uint32_t)xr[q] - 1u];
}

int sm_count_here() {
    int dev = 0, sms = 0;
    PGB_CUDA(cudaGetDevice(&dev));
    PGB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    return sms;
}

}  // namespace

}  // namespace pgb

using namespace pgb;

extern "C" {

int pgb_k4_count(const pgb_blocks* b, void* stream, uint64_t* total) {
    return guard([&] {
        if (!b || !total) fail(PGB_E_INVAL, "NULL argument");
        if (b->offloaded) fail(PGB_E_STATE, "pattern counts need resident blocks (not offloaded)");
        cudaStream_t s = (cudaStream_t)stream;
        const int grid = sm_count_here() * 8;
        DevBuf<unsigned long long> part(grid, s), out(1, s);
        k_k4<<<grid, kPatThreads, 0, s>>>(b->rowptr.ptr, b->rowidx.ptr, b->col.ptr, (uint32_t)b->m, part.ptr);
        PGB_CHECK_LAUNCH("k_k4");
        k_sum_u64<<<1, 256, 0, s>>>(part.ptr, (uint32_t)grid, out.ptr);
        PGB_CHECK_LAUNCH("k_sum_u64");
        unsigned long long h = 0;
        PGB_CUDA(cudaMemcpyAsync(&h, out.ptr, 8, cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaStreamSynchronize(s));
        *total = h;
    });
}

int pgb_c4_count(const pgb_blocks* b, void* stream, uint64_t* total) {
    return guard([&] {
        if (!b || !total) fail(PGB_E_INVAL, "NULL argument");
        if (b->offloaded) fail(PGB_E_STATE, "pattern counts need resident blocks (not offloaded)");
        cudaStream_t s = (cudaStream_t)stream;
        const uint32_t n = b->n;
        const uint64_t m = b->m;
        if (n == 0 || m == 0) {
            *total = 0;
            return;
        }
        // one counter array of n words per CTA, padded to 256 bytes; as many
        // CTAs as the budget holds, at most two per SM
        const uint64_t stride = ((uint64_t)n + 63) / 64 * 64;
        const uint64_t fit = kC4CounterBudget / (stride * 4);
        const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(fit, (uint64_t)sm_count_here() * 2));
        DevBuf<uint32_t> itail(m, s), counters(stride * grid, s);
        DevBuf<unsigned long long> part(grid, s), out(1, s);
        DevBuf<unsigned int> cursor(1, s);
        k_tails_of<<<(unsigned)std::min<uint64_t>((m + 255) / 256, 148ull * 32), 256, 0, s>>>(b->xr.ptr,
                                                                                            b->rowidx.ptr, m, itail.ptr);
        PGB_CHECK_LAUNCH("k_tails_of");
        PGB_CUDA(cudaMemsetAsync(counters.ptr, 0, counters.bytes(), s));
        PGB_CUDA(cudaMemsetAsync(cursor.ptr, 0, 4, s));
        k_c4<<<grid, kC4Threads, 0, s>>>(b->rowptr.ptr, b->col.ptr, b->colptr.ptr, itail.ptr, n, counters.ptr, stride,
                                         cursor.ptr, part.ptr);
        PGB_CHECK_LAUNCH("k_c4");
        k_sum_u64<<<1, 256, 0, s>>>(part.ptr, (uint32_t)grid, out.ptr);
        PGB_CHECK_LAUNCH("k_sum_u64");
        unsigned long long h = 0;
        PGB_CUDA(cudaMemcpyAsync(&h, out.ptr, 8, cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaStreamSynchronize(s));
        *total = h;
    });
}

}  // extern "C"
