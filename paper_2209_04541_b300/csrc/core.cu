// Dense count of the top block of the degree order.
//
// In the degree order the highest ranks hold the hubs, and the block of the
// top K ranks, A_top = A[c0:n, c0:n] (c0 = n - K), is dense (at R-MAT scale
// 24, 16,384 ranks hold 17 M of the 260 M edges: 12.7% of the block's
// pairs).  A triangle with all three vertices in it is counted here instead
// of by the intersection kernels, as the split of vertices into high- and
// low-degree ones of Alon, Yuster and Zwick ("Finding and counting given
// length cycles", 1997) does: with A the block's symmetric 0/1 adjacency,
// (A·A)[x][y] is the number of common neighbours of x and y inside the
// block, so
//     S[x] = sum_y A[x][y] (A·A)[x][y] = 2 t_top[x]
// (a triangle at x is seen from both of its edges at x), and the block's
// triangle total is sum_x S[x] / 6.  The product is a plain dense GEMM on the
// tensor cores: fp16 0/1 inputs, fp32 accumulation, exact because every
// partial sum is an integer below 2^24 (at most K <= 32,768).  Only the
// column strips on and above the diagonal are formed (A·A is symmetric):
// strip I holds rows [I T, I T + T) and columns [I T, K); its masked row
// sums go to S of its rows, and outside the diagonal block its masked
// column sums go to S of its columns.
//
// The intersection kernels skip every in-edge (u, v) whose tail u is in the
// block (tail row at CSR position >= rowptr[c0]): then v > u and every third
// vertex w > v are in the block too, so those are exactly the block's
// triangles, and every other triangle is still counted once by them.
//
// The block size comes from the autotuner: the lookups the block would take
// from the intersection kernels (per 1,024-rank band of tail ranks, summed at
// partition time) against the GEMM's flops, both turned into time by
// measured rates (constants below).
#include <cublas_v2.h>

#include <algorithm>

#include "core.cuh"

namespace pgb {

namespace {

constexpr uint32_t kTile = 2048;          // rows per strip
constexpr uint32_t kReduceRows = 256;     // rows per CTA of the masked reduction (one per thread)
constexpr uint32_t kReduceCols = 64;      // columns per CTA
// Autotuner rates (B300, R-MAT scale 24, blocks of 8,192 to 24,576 ranks):
// the intersection kernels' time fell by 1.02e-12 to 1.05e-12 s per lookup
// left to the block, and the strips with fill and reduction ran at 0.9-1.6
// PFLOP/s (larger blocks faster; the model's 1.4e15 matched 16,384 ranks
// within 2%).
constexpr double kSecondsPerLookup = 1.0e-12;
constexpr double kGemmFlops = 1.4e15;
constexpr double kMinGainSeconds = 3e-4;

// The block's adjacency from its rows: row r in [c0, n) holds only columns
// in the block (they exceed r), written both ways.  One thread per row: the
// top ranks' rows are short.
__global__ void k_core_fill(const uint32_t* __restrict__ rowptr, const uint32_t* __restrict__ col, uint32_t c0,
                            uint32_t K, __half* __restrict__ A) {
    const __half one = __ushort_as_half((unsigned short)0x3C00u);
    for (uint32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < K; a += gridDim.x * blockDim.x) {
        const uint32_t q1 = rowptr[c0 + a + 1];
        for (uint32_t q = rowptr[c0 + a]; q < q1; ++q) {
            const uint32_t b = col[q] - c0;
            A[(uint64_t)a * K + b] = one;
            A[(uint64_t)b * K + a] = one;
        }
    }
}

// Masked sums of strip rows [r0, r0 + rows) x columns [r0, K) of A·A, held
// column-major in C (leading dimension T): thread t takes row r0 + x (x =
// blockIdx.x * kReduceRows + t) over the CTA's kReduceCols columns; row sums
// go to S[r0 + x], column sums (columns outside the diagonal block) to
// S[column] after a warp and a CTA reduction.
__global__ void __launch_bounds__(kReduceRows)
    k_core_reduce(const __half* __restrict__ A, const float* __restrict__ C, uint32_t K, uint32_t T, uint32_t r0,
                  uint32_t rows, unsigned long long* __restrict__ S) {
    __shared__ unsigned int s_col[kReduceCols];
    const uint32_t x = blockIdx.x * kReduceRows + threadIdx.x;
    const uint32_t y0 = blockIdx.y * kReduceCols, ncols = K - r0;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < kReduceCols) s_col[threadIdx.x] = 0;
    __syncthreads();
    unsigned int rsum = 0;
    for (uint32_t j = 0; j < kReduceCols && y0 + j < ncols; ++j) {
        const uint32_t y = y0 + j;  // column r0 + y of A·A
        unsigned int v = 0;
        if (x < rows && __half2float(A[(uint64_t)(r0 + y) * K + r0 + x]) != 0.0f)
            v = (unsigned int)C[(uint64_t)y * T + x];
        rsum += v;
        if (y >= rows) {  // outside the diagonal block: also a column sum
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0 && v) atomicAdd(&s_col[j], v);
        }
    }
    if (x < rows && rsum) atomicAdd(S + r0 + x, (unsigned long long)rsum);
    __syncthreads();
    if (threadIdx.x < kReduceCols && y0 + threadIdx.x < ncols && s_col[threadIdx.x])
        atomicAdd(S + r0 + y0 + threadIdx.x, (unsigned long long)s_col[threadIdx.x]);
}

// t[c0 + x] += S[x] / 2 (rank space) and *slot = sum S / 6 (one CTA).
__global__ void k_core_finish(const unsigned long long* __restrict__ S, uint32_t K, uint32_t c0,
                              unsigned long long* __restrict__ tv, unsigned long long* __restrict__ slot) {
    __shared__ unsigned long long red[32];
    unsigned long long acc = 0;
    for (uint32_t x = threadIdx.x; x < K; x += blockDim.x) {
        const unsigned long long v = S[x];
        acc += v;
        if (tv && v) atomicAdd(tv + c0 + x, v / 2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) *slot = acc / 6;
    }
}

// Lookups of the in-edges whose tail is among the top kCoreBands bands of
// ranks, per band.  The in-edges with tail u are the edges of u's row, and
// the one at row position i looks up the L_u - 1 - i entries after it, so
// u's in-edges take L_u (L_u - 1) / 2 lookups (L_u = |row u|): one thread per
// top row, a block histogram, one atomic per band.
__global__ void k_core_bands(const uint32_t* __restrict__ rowptr, uint32_t n, uint32_t top,
                             unsigned long long* __restrict__ bands) {
    __shared__ unsigned long long h[kCoreBands];
    if (threadIdx.x < kCoreBands) h[threadIdx.x] = 0;
    __syncthreads();
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < top; i += gridDim.x * blockDim.x) {
        const uint32_t u = n - 1 - i;
        const unsigned long long L = rowptr[u + 1] - rowptr[u];
        if (L > 1) atomicAdd(&h[i / kCoreBand], L * (L - 1) / 2);
    }
    __syncthreads();
    if (threadIdx.x < kCoreBands && h[threadIdx.x]) atomicAdd(bands + threadIdx.x, h[threadIdx.x]);
}

__global__ void k_core_add(const unsigned long long* __restrict__ from, unsigned long long* __restrict__ to) {
    *to += *from;
}

}  // namespace

void core_add_total(const unsigned long long* from, unsigned long long* to, cudaStream_t s) {
    k_core_add<<<1, 1, 0, s>>>(from, to);
    PGB_CHECK_LAUNCH("k_core_add");
}

// A cuBLAS handle per host thread (never destroyed: a handle torn down at
// thread exit could outlive the CUDA context).
static cublasHandle_t blas_handle() {
    static thread_local cublasHandle_t h = nullptr;
    if (!h) {
        if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) {
            h = nullptr;
            fail(PGB_E_CUDA, "cublasCreate failed");
        }
    }
    return h;
}

static void blas_check(cublasStatus_t st, const char* what) {
    if (st != CUBLAS_STATUS_SUCCESS)
        fail(PGB_E_CUDA, std::string(what) + " failed (cuBLAS status " + std::to_string((int)st) + ")");
}

double core_flop(uint32_t K) {
    double macs = 0;
    const uint32_t T = std::min(kTile, K);
    for (uint32_t r0 = 0; r0 < K; r0 += T) macs += (double)std::min(T, K - r0) * (K - r0) * K;
    return 2.0 * macs;
}

// Seconds the dense count of the top K ranks would take (GEMM strips,
// masked reduction of fp16 masks and fp32 strips, fill).
static double core_cost(uint32_t K) {
    const double cells = core_flop(K) / (2.0 * K);
    return core_flop(K) / kGemmFlops + 6.0 * cells / 5e12 + 2.0 * (double)K * K / 5e12 + 5e-5;
}

uint32_t choose_core(const pgb_blocks* b, int32_t opt) {
    if (opt < 0 || b->n == 0) return 0;
    if (opt > 0) {
        const uint64_t k = ((uint64_t)opt + 255) / 256 * 256;
        return (uint32_t)std::min<uint64_t>(k, b->n);
    }
    if (b->core_probes.size() < kCoreBands) return 0;
    uint32_t best = 0;
    double best_gain = kMinGainSeconds;
    for (uint32_t K = kTile; K <= kCoreBands * kCoreBand && K <= b->n; K += kTile) {
        double saved = 0;
        for (uint32_t i = 0; i < K / kCoreBand; ++i) saved += (double)b->core_probes[i];
        const double gain = saved * kSecondsPerLookup - core_cost(K);
        if (gain > best_gain) {
            best_gain = gain;
            best = K;
        }
    }
    return best;
}

void core_band_probes(const pgb_blocks* b, unsigned long long* bands, cudaStream_t s) {
    if (b->m == 0 || b->n == 0) return;
    const uint32_t top = std::min<uint32_t>(b->n, kCoreBands * kCoreBand);
    k_core_bands<<<(top + 255) / 256, 256, 0, s>>>(b->rowptr.ptr, b->n, top, bands);
    PGB_CHECK_LAUNCH("k_core_bands");
}

// cuBLAS workspace of a plan: 32 MiB (its recommendation on this GPU) for
// blocks of 8,192 ranks or more, 4 MiB below.
static uint64_t core_workspace(uint32_t K) { return K >= 8192 ? (32u << 20) : (4u << 20); }

uint64_t core_bytes(uint32_t K) {
    const uint64_t T = std::min(kTile, K);
    return (uint64_t)K * K * sizeof(__half) + T * K * sizeof(float) + (uint64_t)K * 8 + core_workspace(K);
}

void core_prepare(const pgb_blocks* b, uint32_t K, cudaStream_t s, CorePlan& P) {
    P.K = K;
    P.c0 = b->n - K;
    P.m = b->m;
    P.rowptr = b->rowptr.ptr;
    P.col = b->col.ptr;
    P.tile = std::min(kTile, K);
    uint32_t e0 = 0;
    PGB_CUDA(cudaMemcpyAsync(&e0, b->rowptr.ptr + P.c0, 4, cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaStreamSynchronize(s));
    P.e0 = e0;
    P.A.alloc((size_t)K * K, s);
    P.C.alloc((size_t)P.tile * K, s);
    P.S.alloc(K, s);
    P.workspace.alloc(core_workspace(K), s);
}

void core_enqueue(const CorePlan& P, unsigned long long* tv, unsigned long long* slot, cudaStream_t s) {
    const uint32_t K = P.K, T = P.tile;
    PGB_CUDA(cudaMemsetAsync(P.A.ptr, 0, (size_t)K * K * sizeof(__half), s));
    PGB_CUDA(cudaMemsetAsync(P.S.ptr, 0, (size_t)K * 8, s));
    if (P.m > P.e0) {
        k_core_fill<<<(K + 255) / 256, 256, 0, s>>>(P.rowptr, P.col, P.c0, K, P.A.ptr);
        PGB_CHECK_LAUNCH("k_core_fill");
    }
    cublasHandle_t h = blas_handle();
    blas_check(cublasSetStream(h, s), "cublasSetStream");
    blas_check(cublasSetWorkspace(h, P.workspace.ptr, P.workspace.bytes()), "cublasSetWorkspace");
    const float one = 1.0f, zero = 0.0f;
    for (uint32_t r0 = 0; r0 < K; r0 += T) {
        const uint32_t rows = std::min(T, K - r0), cols = K - r0;
        // C[x + y T] = sum_k A[r0 + x][k] A[k][r0 + y]  (A column-major, leading dimension K)
        blas_check(cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_N, (int)rows, (int)cols, (int)K, &one, P.A.ptr + r0,
                                CUDA_R_16F, (int)K, P.A.ptr + (size_t)r0 * K, CUDA_R_16F, (int)K, &zero, P.C.ptr,
                                CUDA_R_32F, (int)T, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT),
                   "cublasGemmEx");
        const dim3 grid((rows + kReduceRows - 1) / kReduceRows, (cols + kReduceCols - 1) / kReduceCols);
        k_core_reduce<<<grid, kReduceRows, 0, s>>>(P.A.ptr, P.C.ptr, K, T, r0, rows, P.S.ptr);
        PGB_CHECK_LAUNCH("k_core_reduce");
    }
    k_core_finish<<<1, 1024, 0, s>>>(P.S.ptr, K, P.c0, tv, slot);
    PGB_CHECK_LAUNCH("k_core_finish");
}

}  // namespace pgb
