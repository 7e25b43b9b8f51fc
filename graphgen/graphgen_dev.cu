// Seeded synthetic graph generators on the device.
//
// The same graphs as graphgen.c, edge for edge and in the same order, written
// straight into device arrays, so that large inputs (the serving mix's jobs
// up to R-MAT scale 22) need neither host generation nor a host copy.  Input
// plumbing only: nothing here belongs to the triangle-counting method, and
// the library under test never calls it.
//
// The stream, the R-MAT edge step and the Feistel relabelling come from
// gg_stream.h, shared with the host generators.  Relabelling by the
// Fisher-Yates permutation (a sequential walk) is taken as a device array of
// the permutation, made on the host.  The random geometric graph repeats the
// host's arithmetic in IEEE double with explicit round-to-nearest operations
// (no fused multiply-add), so each distance test decides as on the host.
//
// Every call runs on the given stream and returns 0, or a negative value for
// bad arguments (-1) or a CUDA error (-3).
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "gg_stream.h"

namespace {

constexpr int kThreads = 256;

unsigned grid_for(uint64_t items) {
    uint64_t g = (items + kThreads - 1) / kThreads;
    if (g > 148ull * 64) g = 148ull * 64;
    return g < 1 ? 1u : (unsigned)g;
}

int bits_of(uint64_t x) {
    int b = 0;
    while (b < 64 && (x >> b) != 0) ++b;
    return b < 1 ? 1 : b;
}

__global__ void k_rmat(uint32_t scale, uint64_t m, uint64_t key, uint64_t ta, uint64_t tb, uint64_t tc, int relabel,
                       uint64_t fkey, const uint32_t* __restrict__ perm, uint32_t* __restrict__ src,
                       uint32_t* __restrict__ dst) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        uint32_t s, d;
        gg_rmat_edge(key, scale, e, ta, tb, tc, &s, &d);
        if (relabel == 1) {
            s = perm[s];
            d = perm[d];
        } else if (relabel == 2) {
            s = gg_feistel(s, scale, fkey);
            d = gg_feistel(d, scale, fkey);
        }
        src[e] = s;
        dst[e] = d;
    }
}

__global__ void k_er_pairs(uint32_t n, uint64_t m, uint64_t key, uint32_t* __restrict__ src,
                           uint32_t* __restrict__ dst) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const uint64_t x = gg_draw(key, e);
        src[e] = gg_below((uint32_t)(x >> 32), n);
        dst[e] = gg_below((uint32_t)x, n);
    }
}

// Random geometric graph: points, their grid cells, and cell histogram.
__global__ void k_rgg_points(uint32_t n, uint64_t key, uint32_t g, double* __restrict__ px, double* __restrict__ py,
                             uint32_t* __restrict__ cell, uint32_t* __restrict__ ids, uint32_t* __restrict__ hist) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t x = gg_draw(key, i);
        const double fx = __dmul_rn((double)(uint32_t)(x >> 32), 1.0 / 4294967296.0);
        const double fy = __dmul_rn((double)(uint32_t)x, 1.0 / 4294967296.0);
        uint32_t cx = (uint32_t)__dmul_rn(fx, (double)g), cy = (uint32_t)__dmul_rn(fy, (double)g);
        if (cx >= g) cx = g - 1;
        if (cy >= g) cy = g - 1;
        px[i] = fx;
        py[i] = fy;
        cell[i] = cy * g + cx;
        ids[i] = i;
        atomicAdd(&hist[cell[i]], 1u);
    }
}

// Neighbours b > a of point a within distance r, visited in the host's
// order (cell rows dy = -1..1, columns dx = -1..1, points of a cell by
// ascending index); `emit` sees each one.
template <class F>
__device__ void rgg_visit(uint32_t a, uint32_t g, double r2, const double* __restrict__ px,
                          const double* __restrict__ py, const uint32_t* __restrict__ cell,
                          const uint32_t* __restrict__ start, const uint32_t* __restrict__ order, F&& emit) {
    const int64_t cx = cell[a] % g, cy = cell[a] / g;
    const double ax = px[a], ay = py[a];
    for (int64_t dy = -1; dy <= 1; ++dy) {
        for (int64_t dx = -1; dx <= 1; ++dx) {
            const int64_t nx = cx + dx, ny = cy + dy;
            if (nx < 0 || ny < 0 || nx >= g || ny >= g) continue;
            const uint64_t k = (uint64_t)ny * g + nx;
            for (uint32_t t = start[k]; t < start[k + 1]; ++t) {
                const uint32_t b = order[t];
                if (b <= a) continue;
                const double ddx = __dsub_rn(ax, px[b]), ddy = __dsub_rn(ay, py[b]);
                if (__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)) < r2) emit(b);
            }
        }
    }
}

__global__ void k_rgg_count(uint32_t n, uint32_t g, double r2, const double* __restrict__ px,
                            const double* __restrict__ py, const uint32_t* __restrict__ cell,
                            const uint32_t* __restrict__ start, const uint32_t* __restrict__ order,
                            uint64_t* __restrict__ deg) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += stride) {
        uint64_t c = 0;
        rgg_visit(a, g, r2, px, py, cell, start, order, [&](uint32_t) { ++c; });
        deg[a] = c;
    }
}

__global__ void k_rgg_fill(uint32_t n, uint32_t g, double r2, const double* __restrict__ px,
                           const double* __restrict__ py, const uint32_t* __restrict__ cell,
                           const uint32_t* __restrict__ start, const uint32_t* __restrict__ order,
                           const uint64_t* __restrict__ off, uint32_t* __restrict__ src, uint32_t* __restrict__ dst) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += stride) {
        uint64_t o = off[a];
        rgg_visit(a, g, r2, px, py, cell, start, order, [&](uint32_t b) {
            src[o] = a;
            dst[o] = b;
            ++o;
        });
    }
}

struct RggPlan {
    uint32_t n = 0, g = 0;
    double r2 = 0;
    uint64_t ncell = 0;
    double *px = nullptr, *py = nullptr;
    uint32_t *cell = nullptr, *order = nullptr, *start = nullptr;
    uint64_t* off = nullptr;
    int64_t count = 0;
};

template <class T>
cudaError_t alloc(T** p, uint64_t count, cudaStream_t s) {
    return cudaMallocAsync(reinterpret_cast<void**>(p), (count ? count : 1) * sizeof(T), s);
}

void release(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

void plan_release(RggPlan* P, cudaStream_t s) {
    release(P->px, s);
    release(P->py, s);
    release(P->cell, s);
    release(P->order, s);
    release(P->start, s);
    release(P->off, s);
    delete P;
}

}  // namespace

#define GGD_TRY(x)                        \
    do {                                  \
        if ((x) != cudaSuccess) {         \
            cudaGetLastError();           \
            return -3;                    \
        }                                 \
    } while (0)

extern "C" {

// R-MAT with m raw edges on 2^scale vertices, as gg_rmat: relabel 0 none,
// 1 through `perm` (a device array of 2^scale labels, e.g. the host's
// Fisher-Yates permutation), 2 the Feistel bijection.
int ggd_rmat(uint32_t scale, uint64_t m, double a, double b, double c, uint64_t seed, int relabel,
             const uint32_t* perm, uint32_t* src, uint32_t* dst, void* stream) {
    if (scale == 0 || scale > 31 || a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return -1;
    if (relabel < 0 || relabel > 2 || (relabel == 1 && !perm) || (m && (!src || !dst))) return -1;
    if (!m) return 0;
    uint64_t ta, tb, tc;
    gg_rmat_thresholds(a, b, c, &ta, &tb, &tc);
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_rmat<<<grid_for(m), kThreads, 0, s>>>(scale, m, gg_mix(seed), ta, tb, tc, relabel,
                                            gg_mix(seed ^ GG_TAG_FEISTEL), perm, src, dst);
    GGD_TRY(cudaGetLastError());
    return 0;
}

// m i.i.d. uniform ordered pairs over [0, n)^2, as gg_er_pairs.
int ggd_er_pairs(uint32_t n, uint64_t m, uint64_t seed, uint32_t* src, uint32_t* dst, void* stream) {
    if (n == 0 || (m && (!src || !dst))) return -1;
    if (!m) return 0;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_er_pairs<<<grid_for(m), kThreads, 0, s>>>(n, m, gg_mix(seed ^ 0x4552ULL), src, dst);
    GGD_TRY(cudaGetLastError());
    return 0;
}

// Random geometric graph, as gg_rgg, in two steps: the plan places the
// points and counts the edges (*count, synchronising the stream); fill
// writes them; free releases the plan (stream-ordered).
int ggd_rgg_plan(uint32_t n, double r, uint64_t seed, void* stream, void** plan, int64_t* count) {
    if (!plan || !count || !(r > 0.0)) return -1;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    RggPlan* P = new RggPlan();
    P->n = n;
    uint32_t g = (uint32_t)floor(1.0 / r);
    if (g < 1) g = 1;
    if (g > 65536) g = 65536;
    P->g = g;
    P->r2 = r * r;
    P->ncell = (uint64_t)g * g;
    if (P->ncell >= (1ull << 31)) {
        delete P;
        return -1;
    }
    *plan = P;
    *count = 0;
    if (n == 0) return 0;
    const uint64_t key = gg_mix(seed ^ 0x524747ULL);
    uint32_t *cell_sorted = nullptr, *ids = nullptr, *hist = nullptr;
    uint64_t* deg = nullptr;
    void* tmp = nullptr;
    size_t t1 = 0, t2 = 0, t3 = 0;
    const int bits = bits_of(P->ncell - 1);
    auto fail = [&] {
        cudaGetLastError();
        release(cell_sorted, s);
        release(ids, s);
        release(hist, s);
        release(deg, s);
        release(tmp, s);
        plan_release(P, s);
        *plan = nullptr;
        return -3;
    };
    if (alloc(&P->px, n, s) || alloc(&P->py, n, s) || alloc(&P->cell, n, s) || alloc(&P->order, n, s) ||
        alloc(&P->start, P->ncell + 1, s) || alloc(&P->off, (uint64_t)n + 1, s) || alloc(&cell_sorted, n, s) ||
        alloc(&ids, n, s) || alloc(&hist, P->ncell + 1, s) || alloc(&deg, (uint64_t)n + 1, s))
        return fail();
    if (cudaMemsetAsync(hist, 0, (P->ncell + 1) * 4, s)) return fail();
    k_rgg_points<<<grid_for(n), kThreads, 0, s>>>(n, key, g, P->px, P->py, P->cell, ids, hist);
    if (cudaGetLastError()) return fail();
    // points by cell, ascending index within a cell (the sort is stable)
    if (cub::DeviceRadixSort::SortPairs(nullptr, t1, P->cell, cell_sorted, ids, P->order, (int64_t)n, 0, bits, s))
        return fail();
    if (cub::DeviceScan::ExclusiveSum(nullptr, t2, hist, P->start, (int64_t)P->ncell + 1, s)) return fail();
    if (cub::DeviceScan::ExclusiveSum(nullptr, t3, deg, P->off, (int64_t)n + 1, s)) return fail();
    const size_t tb = t1 > t2 ? (t1 > t3 ? t1 : t3) : (t2 > t3 ? t2 : t3);
    if (cudaMallocAsync(&tmp, tb ? tb : 1, s)) return fail();
    if (cub::DeviceRadixSort::SortPairs(tmp, t1, P->cell, cell_sorted, ids, P->order, (int64_t)n, 0, bits, s))
        return fail();
    if (cub::DeviceScan::ExclusiveSum(tmp, t2, hist, P->start, (int64_t)P->ncell + 1, s)) return fail();
    k_rgg_count<<<grid_for(n), kThreads, 0, s>>>(n, g, P->r2, P->px, P->py, P->cell, P->start, P->order, deg);
    if (cudaGetLastError()) return fail();
    if (cudaMemsetAsync(deg + n, 0, 8, s)) return fail();
    if (cub::DeviceScan::ExclusiveSum(tmp, t3, deg, P->off, (int64_t)n + 1, s)) return fail();
    uint64_t total = 0;
    if (cudaMemcpyAsync(&total, P->off + n, 8, cudaMemcpyDeviceToHost, s)) return fail();
    if (cudaStreamSynchronize(s)) return fail();
    release(cell_sorted, s);
    release(ids, s);
    release(hist, s);
    release(deg, s);
    release(tmp, s);
    P->count = (int64_t)total;
    *count = P->count;
    return 0;
}

int ggd_rgg_fill(void* plan, uint32_t* src, uint32_t* dst, void* stream) {
    RggPlan* P = static_cast<RggPlan*>(plan);
    if (!P || (P->count && (!src || !dst))) return -1;
    if (!P->count) return 0;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_rgg_fill<<<grid_for(P->n), kThreads, 0, s>>>(P->n, P->g, P->r2, P->px, P->py, P->cell, P->start, P->order,
                                                   P->off, src, dst);
    GGD_TRY(cudaGetLastError());
    return 0;
}

void ggd_rgg_free(void* plan, void* stream) {
    if (plan) plan_release(static_cast<RggPlan*>(plan), static_cast<cudaStream_t>(stream));
}

}  // extern "C"
