// Allocation-free triangle count over a caller-built oriented graph.
//
// The paper has no counterpart to this entry point.  It serves callers that
// must not allocate device memory while they run: programs whose host
// framework hands out every byte of device memory from its own pool and
// forbids other allocations, and latency-critical loops that cannot afford
// the device-wide synchronisation that cudaMalloc / cudaFree can cause.
//
// Instead of buffers from the library allocator, this variant of the
// counting kernel keeps its working memory (a work cursor, one partial count
// per CTA, and a rank-space per-vertex accumulator) in one fixed file-scope
// device array.  The array lives as long as the library is loaded, on every
// GPU that loads it.  Host code must not pass the array's name to a kernel
// (on the host that name is only a stand-in); it obtains the device address
// once per device with cudaGetSymbolAddress and passes that.
#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace pgb {
namespace {

constexpr uint32_t kNoAllocMaxVertices = PGB_NOALLOC_MAX_VERTICES;  // accumulator entries
constexpr int kNoAllocMaxCtas = 2048;                // per-CTA partial slots
constexpr int kNaThreads = 256;
constexpr int kNaWarps = kNaThreads / 32;
constexpr uint32_t kNaChunk = 64;                    // edges per dequeued chunk
constexpr unsigned kNaFull = 0xffffffffu;
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
    unsigned long long tv[kNoAllocMaxVertices];   // per-vertex counts by rank
    unsigned long long partials[kNoAllocMaxCtas]; // per-CTA totals
    unsigned int seen[kNoAllocMaxVertices / 32];  // perm targets written (one bit each)
    unsigned long long cursor;                    // next edge chunk
    unsigned int error;                           // error bits (kNaErr*)
};

// Error bits: which rule of the input contract a call's graph broke.
constexpr unsigned kNaErrRange = 1u;     // an offset, column or perm entry out of range
constexpr unsigned kNaErrOrder = 2u;     // offsets decreasing, or a row not strictly ascending above u
constexpr unsigned kNaErrPerm = 4u;      // perm maps two ranks to one vertex

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Zero what must start at zero: the first n accumulator entries, the perm
// bitmap's first ceil(n / 32) words, the cursor and the error word
// (partials are overwritten, not accumulated).
__global__ void k_na_clear(NoAllocScratch* __restrict__ s, uint32_t n) {
    uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) s->tv[i] = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < (n + 31) / 32; i += stride) s->seen[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s->cursor = 0;
        s->error = 0;
    }
}

__device__ __forceinline__ uint32_t na_lower_bound(const uint32_t* __restrict__ a, uint32_t b, uint32_t e,
                                                   uint32_t x) {
    uint32_t len = e - b;
    while (len > 0) {
        uint32_t half = len >> 1;
        if (__ldg(a + b + half) < x) {
            b += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return b;
}

// Row of edge e: the largest u in [0, n) with rowptr[u] <= e.
__device__ __forceinline__ uint32_t na_row_of(const uint32_t* __restrict__ rowptr, uint32_t n, uint32_t e) {
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(rowptr + mid) <= e) lo = mid; else hi = mid;
    }
    return lo;
}

// Persistent counting kernel, binary-search intersection with the work of
// 32 edges flattened across the warp (the same arithmetic as the library's
// main kernel, over plain CSR edge order).  Malformed offsets or columns
// set the error bit and the edge is skipped, so no read leaves the arrays.
template <bool PV>
__global__ void __launch_bounds__(kNaThreads)
    k_na_count(uint32_t n, uint32_t m, const uint32_t* __restrict__ rowptr, const uint32_t* __restrict__ col,
               NoAllocScratch* __restrict__ s) {
    __shared__ uint32_t s_edge[kNaWarps][32];
    __shared__ unsigned long long s_red[kNaWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    s_edge[warp][lane] = 0;
    __syncwarp();
    unsigned long long cnt = 0;
    const unsigned long long nchunks = ((unsigned long long)m + kNaChunk - 1) / kNaChunk;
    while (true) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(&s->cursor, 1ull);
        c = __shfl_sync(kNaFull, c, 0);
        if (c >= nchunks) break;
        const unsigned long long i0 = c * kNaChunk;
        const unsigned long long end = min(i0 + kNaChunk, (unsigned long long)m);
        for (unsigned long long i = i0; i < end; i += 32) {
            const bool active = i + lane < end;
            const uint32_t e = (uint32_t)(i + lane);
            uint32_t sb = 0, sl = 0, lb = 0, ll = 0, u = 0, v = 0;
            bool ok = false;
            if (active) {
                u = na_row_of(rowptr, n, e);
                v = __ldg(col + e);
                uint32_t xe = __ldg(rowptr + u + 1);
                if (v < n && xe <= m && e < xe) {
                    uint32_t yb = __ldg(rowptr + v), ye = __ldg(rowptr + v + 1);
                    if (yb <= ye && ye <= m) {
                        ok = true;
                        const uint32_t xb = e + 1;
                        const uint32_t lx = xe - xb, ly = ye - yb;
                        if (lx <= ly) {
                            sb = xb; sl = lx; lb = yb; ll = ly;
                        } else {
                            sb = yb; sl = ly; lb = xb; ll = lx;
                        }
                        if (ll == 0) sl = 0;
                    }
                }
                if (!ok) atomicOr(&s->error, kNaErrRange);
            }
            uint32_t incl = sl;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(kNaFull, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t total = __shfl_sync(kNaFull, incl, 31);
            const uint32_t excl = incl - sl;
            for (uint32_t base = 0; base < total; base += 32) {
                const uint32_t f = base + lane;
                int o = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    uint32_t ex = __shfl_sync(kNaFull, excl, o + step);
                    if (ex <= f) o += step;
                }
                const uint32_t o_ex = __shfl_sync(kNaFull, excl, o);
                const uint32_t o_sb = __shfl_sync(kNaFull, sb, o);
                const uint32_t o_lb = __shfl_sync(kNaFull, lb, o);
                const uint32_t o_ll = __shfl_sync(kNaFull, ll, o);
                if (f < total) {
                    const uint32_t x = __ldg(col + o_sb + (f - o_ex));
                    const uint32_t lend = o_lb + o_ll;
                    const uint32_t p = na_lower_bound(col, o_lb, lend, x);
                    if (p < lend && __ldg(col + p) == x) {
                        ++cnt;
                        if (PV && x < n) {
                            atomicAdd(&s->tv[x], 1ull);
                            atomicAdd(&s_edge[warp][o], 1u);
                        }
                    }
                }
            }
            if (PV) {
                __syncwarp();
                const uint32_t k = s_edge[warp][lane];
                if (k) {
                    atomicAdd(&s->tv[u], (unsigned long long)k);
                    atomicAdd(&s->tv[v], (unsigned long long)k);
                    s_edge[warp][lane] = 0;
                }
                __syncwarp();
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(kNaFull, cnt, o);
    if (lane == 0) s_red[warp] = cnt;
    __syncthreads();
    if (warp == 0) {
        cnt = lane < kNaWarps ? s_red[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(kNaFull, cnt, o);
        if (lane == 0) s->partials[blockIdx.x] = cnt;
    }
}

// Total of the per-CTA partials (one CTA).
__global__ void k_na_reduce(const NoAllocScratch* __restrict__ s, int nparts,
                            unsigned long long* __restrict__ total) {
    __shared__ unsigned long long red[32];
    unsigned long long acc = 0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += s->partials[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kNaFull, acc, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        acc = lane < (int)(blockDim.x >> 5) ? red[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kNaFull, acc, o);
        if (lane == 0) *total = acc;
    }
}

// Per-vertex counts out of the accumulator: by original ID through perm, or
// by rank when perm is NULL.  An out-of-range perm entry, or one that names
// a vertex another rank already took, sets an error bit and is not written.
__global__ void k_na_scatter(NoAllocScratch* __restrict__ s, uint32_t n, const uint32_t* __restrict__ perm,
                             unsigned long long* __restrict__ out) {
    uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        uint32_t dst = perm ? perm[r] : r;
        if (dst >= n) {
            atomicOr(&s->error, kNaErrRange);
            continue;
        }
        if (perm) {
            const unsigned bit = 1u << (dst & 31);
            if (atomicOr(&s->seen[dst >> 5], bit) & bit) {
                atomicOr(&s->error, kNaErrPerm);
                continue;
            }
        }
        out[dst] = s->tv[r];
    }
}

// Header checks: rowptr[0] == 0 and rowptr[n] == m.
__global__ void k_na_check_ends(const uint32_t* __restrict__ rowptr, uint32_t n, uint32_t m,
                                NoAllocScratch* __restrict__ s) {
    if (rowptr[0] != 0 || rowptr[n] != m) atomicOr(&s->error, kNaErrRange);
}

// The ordering contract: offsets non-decreasing (one thread per row), and
// every column above its row and strictly above the previous entry of the
// same row (one thread per edge; with non-decreasing offsets the row found
// by binary search is the edge's own).  Reads stay inside rowptr[0..n] and
// col[0..m); a broken rule only sets an error bit.
__global__ void k_na_check_order(const uint32_t* __restrict__ rowptr, const uint32_t* __restrict__ col,
                                 uint32_t n, uint32_t m, NoAllocScratch* __restrict__ s) {
    const uint32_t stride = gridDim.x * blockDim.x;
    unsigned bad = 0;
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride)
        if (__ldg(rowptr + u) > __ldg(rowptr + u + 1)) bad |= kNaErrOrder;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const uint32_t u = na_row_of(rowptr, n, e);
        const uint32_t v = __ldg(col + e);
        if (v >= n) bad |= kNaErrRange;
        if (v <= u) bad |= kNaErrOrder;
        if (e > __ldg(rowptr + u) && __ldg(col + e - 1) >= v) bad |= kNaErrOrder;
    }
    if (bad) atomicOr(&s->error, bad);
}

std::mutex g_na_mu;
NoAllocScratch* g_na_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device, looked up
// once per device (the first call on a device does it).
NoAllocScratch* scratch_for_current_device() {
    int dev = 0;
    PGB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) fail(PGB_E_INVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            fail(PGB_E_CUDA, std::string("cudaGetSymbolAddress(no-allocation scratch): ") + cudaGetErrorString(e));
        g_na_ptr[dev] = static_cast<NoAllocScratch*>(p);
    }
    return g_na_ptr[dev];
}

}  // namespace
}  // namespace pgb

using namespace pgb;

extern "C" {

int pgb_tc_count_oriented_noalloc(uint32_t n, uint64_t m, const uint32_t* rowptr, const uint32_t* col,
                                  const uint32_t* perm, unsigned long long* total,
                                  unsigned long long* per_vertex, void* stream) {
    return guard([&] {
        if (n > kNoAllocMaxVertices)
            fail(PGB_E_INVAL, "n = " + std::to_string(n) + " exceeds the no-allocation limit of " +
                                  std::to_string(kNoAllocMaxVertices) + " vertices");
        if (m >= (1ull << 32)) fail(PGB_E_OVERFLOW, "m must be below 2^32");
        if (!total) fail(PGB_E_INVAL, "total is NULL");
        if (!rowptr) fail(PGB_E_INVAL, "rowptr is NULL");
        if (m > 0 && !col) fail(PGB_E_INVAL, "col is NULL with m > 0");
        if (m > 0 && n == 0) fail(PGB_E_INVAL, "edges given for an empty vertex set");
        cudaStream_t s = (cudaStream_t)stream;
        NoAllocScratch* sc = scratch_for_current_device();
        int dev = 0, sms = 0, per_sm = 0;
        PGB_CUDA(cudaGetDevice(&dev));
        PGB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const bool pv = per_vertex != nullptr;
        if (pv)
            PGB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_na_count<true>, kNaThreads, 0));
        else
            PGB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_na_count<false>, kNaThreads, 0));
        int grid = std::max(1, per_sm) * std::max(1, sms);
        if (grid > kNoAllocMaxCtas) grid = kNoAllocMaxCtas;

        k_na_clear<<<std::max<uint32_t>(1, std::min<uint32_t>((n + 255) / 256, 1024)), 256, 0, s>>>(sc, n);
        PGB_CHECK_LAUNCH("k_na_clear");
        if (n > 0) {
            k_na_check_ends<<<1, 1, 0, s>>>(rowptr, n, (uint32_t)m, sc);
            PGB_CHECK_LAUNCH("k_na_check_ends");
            const uint64_t work = std::max<uint64_t>(n, m);
            k_na_check_order<<<(uint32_t)std::min<uint64_t>((work + 255) / 256, 4096), 256, 0, s>>>(
                rowptr, col, n, (uint32_t)m, sc);
            PGB_CHECK_LAUNCH("k_na_check_order");
        }
        if (m > 0) {
            if (pv) k_na_count<true><<<grid, kNaThreads, 0, s>>>(n, (uint32_t)m, rowptr, col, sc);
            else k_na_count<false><<<grid, kNaThreads, 0, s>>>(n, (uint32_t)m, rowptr, col, sc);
            PGB_CHECK_LAUNCH("k_na_count");
        } else {
            grid = 0;
        }
        k_na_reduce<<<1, 1024, 0, s>>>(sc, grid, total);
        PGB_CHECK_LAUNCH("k_na_reduce");
        if (pv && n > 0) {
            k_na_scatter<<<std::min<uint32_t>((n + 255) / 256, 1024), 256, 0, s>>>(sc, n, perm, per_vertex);
            PGB_CHECK_LAUNCH("k_na_scatter");
        }
        unsigned int herr = 0;
        PGB_CUDA(cudaMemcpyAsync(&herr, &sc->error, sizeof(herr), cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaStreamSynchronize(s));
        if (herr) {
            std::string why;
            if (herr & kNaErrRange) why += " offsets, columns or perm out of range;";
            if (herr & kNaErrOrder) why += " offsets decreasing, or a row not strictly ascending above its vertex;";
            if (herr & kNaErrPerm) why += " perm maps two ranks to one vertex;";
            fail(PGB_E_INVAL, "malformed oriented graph:" + why);
        }
    });
}

}  // extern "C"
