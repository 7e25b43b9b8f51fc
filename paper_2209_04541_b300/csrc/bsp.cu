// Single-block bulk-synchronous computations on the block store (PGAbB
// Section 3.2: each block-list holds one block and every iteration visits
// every edge): connected components by Shiloach-Vishkin (Section 3.4) and
// PageRank (Section 5.2.1).
//
// Both run on the partition's oriented graph in rank space: every undirected
// edge appears once as an oriented edge (rowidx[e], col[e]); the in-edge index
// gives each vertex its lower-ranked neighbours.
//
// Shiloach-Vishkin.  C[x] is a parent pointer (rank space).  A hook launch
// visits every oriented edge (u, v); when the parents of u and v differ, the
// one with the larger original ID is hooked below the other if it is still
// a root (compare-and-swap, so no hook is lost).  A link launch then points
// every vertex at its root (pointer jumping).  Parents only ever move to a
// smaller original ID, so the trees have no cycles and the root of each
// component is its vertex of smallest original ID: the labels are unique.
// Iterations repeat until a hook launch hooks nothing.
//
// PageRank.  r_t+1(v) = (1 - d) / n + d * sum over neighbours u of
// r_t(u) / deg(u) in double precision, pulled per vertex over its row (upper
// neighbours) and its in-edge tails (lower neighbours): no atomics.  Ranks
// are degree-ordered, so the vertices of degree >= kWarpDegree form one top
// range, summed by one warp each (coalesced loads); the others by one
// thread each.  The L1 change of an iteration is reduced per CTA without
// atomics; the host reads it back after each iteration and stops below the
// tolerance or at the iteration limit.
#include <algorithm>

#include "internal.cuh"

namespace pgb {

namespace {

constexpr int kBspThreads = 256;
constexpr uint32_t kWarpDegree = 64;   // vertices of at least this degree are summed by a warp
constexpr uint32_t kMaxJumps = 1u << 20;  // bound on one vertex's pointer jumps per link launch

int bsp_grid(uint64_t items) {
    int dev = 0, sms = 0;
    PGB_CUDA(cudaGetDevice(&dev));
    PGB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const uint64_t want = (items + kBspThreads - 1) / kBspThreads;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)sms * 16));
}

__global__ void k_cc_init(uint32_t* __restrict__ C, uint32_t n) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) C[v] = v;
}

// Hook: one pass over the oriented edges.  *hooks counts successful hooks
// (one atomic per warp that hooked).
__global__ void k_cc_hook(const uint32_t* __restrict__ rowidx, const uint32_t* __restrict__ col, uint64_t m,
                          const uint32_t* __restrict__ perm, uint32_t* __restrict__ C,
                          unsigned long long* __restrict__ hooks) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint32_t mine = 0;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const uint32_t cu = C[rowidx[e]], cv = C[col[e]];
        if (cu == cv) continue;
        const bool u_hi = __ldg(perm + cu) > __ldg(perm + cv);
        const uint32_t hi = u_hi ? cu : cv, lo = u_hi ? cv : cu;
        // read first: once a root has been hooked, the other edges that would
        // hook it skip the compare-and-swap (a root shared by many edges, such
        // as a giant component's, is contended only until its first hook)
        if (*reinterpret_cast<volatile uint32_t*>(C + hi) != hi) continue;
        if (atomicCAS(C + hi, hi, lo) == hi) ++mine;
    }
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(hooks, (unsigned long long)mine);
}

// Link: every vertex jumps to its root.  A chain longer than kMaxJumps is
// cut there and flagged, and the host repeats the launch; otherwise one
// launch leaves every vertex pointing at a root.
__global__ void k_cc_link(uint32_t* __restrict__ C, uint32_t n, unsigned int* __restrict__ moved) {
    const uint32_t stride = gridDim.x * blockDim.x;
    bool mv = false;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        uint32_t c = C[v];
        uint32_t jumps = 0;
        for (uint32_t cc = C[c]; c != cc && jumps < kMaxJumps; cc = C[c], ++jumps) c = cc;
        if (c != C[v]) C[v] = c;
        if (jumps == kMaxJumps) mv = true;
    }
    if (__any_sync(0xffffffffu, mv) && (threadIdx.x & 31) == 0) atomicOr(moved, 1u);
}

// Labels by original ID: out[perm[v]] = perm[root of v]; counts roots.
__global__ void k_cc_labels(const uint32_t* __restrict__ C, const uint32_t* __restrict__ perm, uint32_t n,
                            uint32_t* __restrict__ out, unsigned long long* __restrict__ roots) {
    const uint32_t stride = gridDim.x * blockDim.x;
    uint32_t mine = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        out[perm[v]] = perm[C[v]];
        mine += C[v] == v;
    }
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(roots, (unsigned long long)mine);
}

// In-edge tails in head order (tail of in-edge q: the row of its edge).
__global__ void k_in_tails(const unsigned long long* __restrict__ xr, const uint32_t* __restrict__ rowidx, uint64_t m,
                           uint32_t* __restrict__ itail) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += stride)
        itail[q] = rowidx[(uint32_t)xr[q] - 1u];
}

// deg[v] (undirected) and the first rank of degree >= kWarpDegree.
__global__ void k_pr_init(const uint32_t* __restrict__ rowptr, const uint32_t* __restrict__ colptr, uint32_t n,
                          double* __restrict__ r, double* __restrict__ c, unsigned int* __restrict__ first_heavy) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint32_t deg = rowptr[v + 1] - rowptr[v] + colptr[v + 1] - colptr[v];
        r[v] = 1.0 / n;
        c[v] = deg ? r[v] / deg : 0.0;
        if (deg >= kWarpDegree && (v == 0 || rowptr[v] - rowptr[v - 1] + colptr[v] - colptr[v - 1] < kWarpDegree))
            atomicMin(first_heavy, v);
    }
}

__device__ __forceinline__ double pr_sum(const uint32_t* __restrict__ col, const uint32_t* __restrict__ itail,
                                         const double* __restrict__ c, uint32_t rb, uint32_t re, uint32_t ib,
                                         uint32_t ie, uint32_t lane, uint32_t step) {
    double s = 0.0;
    for (uint32_t e = rb + lane; e < re; e += step) s += __ldg(c + __ldg(col + e));
    for (uint32_t q = ib + lane; q < ie; q += step) s += __ldg(c + __ldg(itail + q));
    return s;
}

// One PageRank iteration over ranks [v0, v1): thread per vertex (light
// range) or warp per vertex (heavy range).  Writes the new rank and c = r /
// deg, and the CTA's L1 change into part[blockIdx.x].
template <bool kWarp>
__global__ void __launch_bounds__(kBspThreads)
    k_pr_iter(const uint32_t* __restrict__ rowptr, const uint32_t* __restrict__ col,
              const uint32_t* __restrict__ colptr, const uint32_t* __restrict__ itail, uint32_t v0, uint32_t v1,
              uint32_t n, double damping, const double* __restrict__ r, const double* __restrict__ c,
              double* __restrict__ r_out, double* __restrict__ c_out, double* __restrict__ part) {
    __shared__ double red[kBspThreads / 32];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double base = (1.0 - damping) / n;
    double change = 0.0;
    if (kWarp) {
        const uint32_t gw = blockIdx.x * (kBspThreads / 32) + warp, nw = gridDim.x * (kBspThreads / 32);
        for (uint32_t v = v0 + gw; v < v1; v += nw) {
            const uint32_t rb = rowptr[v], re = rowptr[v + 1], ib = colptr[v], ie = colptr[v + 1];
            double s = pr_sum(col, itail, c, rb, re, ib, ie, lane, 32);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) {
                const double nr = base + damping * s;
                const uint32_t deg = re - rb + ie - ib;
                r_out[v] = nr;
                c_out[v] = deg ? nr / deg : 0.0;
                change += fabs(nr - r[v]);
            }
        }
    } else {
        const uint32_t stride = gridDim.x * blockDim.x;
        for (uint32_t v = v0 + blockIdx.x * blockDim.x + threadIdx.x; v < v1; v += stride) {
            const uint32_t rb = rowptr[v], re = rowptr[v + 1], ib = colptr[v], ie = colptr[v + 1];
            const double nr = base + damping * pr_sum(col, itail, c, rb, re, ib, ie, 0, 1);
            const uint32_t deg = re - rb + ie - ib;
            r_out[v] = nr;
            c_out[v] = deg ? nr / deg : 0.0;
            change += fabs(nr - r[v]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) change += __shfl_xor_sync(0xffffffffu, change, o);
    if (lane == 0) red[warp] = change;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kBspThreads / 32; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// Sum of part[0, k) into *out (one CTA), and ranks to original IDs when asked.
__global__ void k_sum_f64(const double* __restrict__ part, uint32_t k, double* __restrict__ out) {
    __shared__ double red[32];
    double s = 0.0;
    for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) s += part[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (uint32_t w = 0; w < (blockDim.x >> 5); ++w) t += red[w];
        *out = t;
    }
}

__global__ void k_scatter_f64(const double* __restrict__ r, const uint32_t* __restrict__ perm, uint32_t n,
                              double* __restrict__ out) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) out[perm[v]] = r[v];
}

void need_resident(const pgb_blocks* b) {
    if (b->offloaded) fail(PGB_E_STATE, "the bulk-synchronous kernels need resident blocks (not offloaded)");
}

}  // namespace

}  // namespace pgb

using namespace pgb;

extern "C" {

int pgb_cc_run(const pgb_blocks* b, void* stream, uint32_t* labels, int mem, uint32_t* iterations,
               uint64_t* components) {
    return guard([&] {
        if (!b || !labels) fail(PGB_E_INVAL, "NULL argument");
        need_resident(b);
        cudaStream_t s = (cudaStream_t)stream;
        const uint32_t n = b->n;
        const uint64_t m = b->m;
        DevBuf<uint32_t> C(std::max<uint32_t>(n, 1), s), out(std::max<uint32_t>(n, 1), s);
        DevBuf<unsigned long long> cnt(2, s);
        DevBuf<unsigned int> moved(1, s);
        k_cc_init<<<bsp_grid(n), kBspThreads, 0, s>>>(C.ptr, n);
        PGB_CHECK_LAUNCH("k_cc_init");
        uint32_t it = 0;
        for (;;) {
            ++it;
            unsigned long long hooks = 0;
            PGB_CUDA(cudaMemsetAsync(cnt.ptr, 0, 8, s));
            if (m) {
                k_cc_hook<<<bsp_grid(m), kBspThreads, 0, s>>>(b->rowidx.ptr, b->col.ptr, m, b->perm.ptr, C.ptr, cnt.ptr);
                PGB_CHECK_LAUNCH("k_cc_hook");
            }
            // link until no vertex moves (one launch unless a chain is very long)
            for (;;) {
                unsigned int mv = 0;
                PGB_CUDA(cudaMemsetAsync(moved.ptr, 0, 4, s));
                k_cc_link<<<bsp_grid(n), kBspThreads, 0, s>>>(C.ptr, n, moved.ptr);
                PGB_CHECK_LAUNCH("k_cc_link");
                PGB_CUDA(cudaMemcpyAsync(&mv, moved.ptr, 4, cudaMemcpyDeviceToHost, s));
                PGB_CUDA(cudaMemcpyAsync(&hooks, cnt.ptr, 8, cudaMemcpyDeviceToHost, s));
                PGB_CUDA(cudaStreamSynchronize(s));
                if (!mv) break;
            }
            if (hooks == 0) break;
        }
        unsigned long long roots = 0;
        PGB_CUDA(cudaMemsetAsync(cnt.ptr + 1, 0, 8, s));
        if (n) {
            k_cc_labels<<<bsp_grid(n), kBspThreads, 0, s>>>(C.ptr, b->perm.ptr, n, out.ptr, cnt.ptr + 1);
            PGB_CHECK_LAUNCH("k_cc_labels");
        }
        PGB_CUDA(cudaMemcpyAsync(&roots, cnt.ptr + 1, 8, cudaMemcpyDeviceToHost, s));
        copy_out(labels, out.ptr, (size_t)n * 4, mem, s);
        PGB_CUDA(cudaStreamSynchronize(s));
        if (iterations) *iterations = it;
        if (components) *components = roots;
    });
}

void pgb_pagerank_opts_default(pgb_pagerank_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->damping = 0.85;
    o->tol = 1e-4;
    o->max_iter = 20;
}

int pgb_pagerank_run(const pgb_blocks* b, const pgb_pagerank_opts* opts, void* stream, double* ranks, int mem,
                     uint32_t* iterations, double* last_change) {
    return guard([&] {
        if (!b || !ranks) fail(PGB_E_INVAL, "NULL argument");
        need_resident(b);
        pgb_pagerank_opts o;
        if (opts) o = *opts; else pgb_pagerank_opts_default(&o);
        if (!(o.damping >= 0.0 && o.damping <= 1.0) || !(o.tol >= 0.0)) fail(PGB_E_INVAL, "bad damping or tol");
        cudaStream_t s = (cudaStream_t)stream;
        const uint32_t n = b->n;
        const uint64_t m = b->m;
        if (n == 0) {
            if (iterations) *iterations = 0;
            if (last_change) *last_change = 0.0;
            return;
        }
        DevBuf<double> r[2] = {DevBuf<double>(n, s), DevBuf<double>(n, s)};
        DevBuf<double> c[2] = {DevBuf<double>(n, s), DevBuf<double>(n, s)};
        DevBuf<uint32_t> itail(std::max<uint64_t>(m, 1), s);
        DevBuf<unsigned int> heavy(1, s);
        if (m) {
            k_in_tails<<<bsp_grid(m), kBspThreads, 0, s>>>(b->xr.ptr, b->rowidx.ptr, m, itail.ptr);
            PGB_CHECK_LAUNCH("k_in_tails");
        }
        PGB_CUDA(cudaMemcpyAsync(heavy.ptr, &n, 4, cudaMemcpyHostToDevice, s));
        k_pr_init<<<bsp_grid(n), kBspThreads, 0, s>>>(b->rowptr.ptr, b->colptr.ptr, n, r[0].ptr, c[0].ptr, heavy.ptr);
        PGB_CHECK_LAUNCH("k_pr_init");
        uint32_t v_heavy = n;
        PGB_CUDA(cudaMemcpyAsync(&v_heavy, heavy.ptr, 4, cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaStreamSynchronize(s));
        const int g_light = bsp_grid(v_heavy);
        const int g_heavy = bsp_grid((uint64_t)(n - v_heavy) * 32);
        DevBuf<double> part((size_t)g_light + g_heavy, s), change(1, s);
        uint32_t it = 0;
        double err = 0.0;
        int cur = 0;
        while (it < o.max_iter) {
            const int nx = cur ^ 1;
            k_pr_iter<false><<<g_light, kBspThreads, 0, s>>>(b->rowptr.ptr, b->col.ptr, b->colptr.ptr, itail.ptr, 0,
                                                            v_heavy, n, o.damping, r[cur].ptr, c[cur].ptr, r[nx].ptr,
                                                            c[nx].ptr, part.ptr);
            k_pr_iter<true><<<g_heavy, kBspThreads, 0, s>>>(b->rowptr.ptr, b->col.ptr, b->colptr.ptr, itail.ptr,
                                                           v_heavy, n, n, o.damping, r[cur].ptr, c[cur].ptr,
                                                           r[nx].ptr, c[nx].ptr, part.ptr + g_light);
            PGB_CHECK_LAUNCHES("k_pr_iter", 2);
            k_sum_f64<<<1, 256, 0, s>>>(part.ptr, (uint32_t)(g_light + g_heavy), change.ptr);
            PGB_CHECK_LAUNCH("k_sum_f64");
            PGB_CUDA(cudaMemcpyAsync(&err, change.ptr, 8, cudaMemcpyDeviceToHost, s));
            PGB_CUDA(cudaStreamSynchronize(s));
            cur = nx;
            ++it;
            if (err < o.tol) break;
        }
        DevBuf<double> out(n, s);
        k_scatter_f64<<<bsp_grid(n), kBspThreads, 0, s>>>(r[cur].ptr, b->perm.ptr, n, out.ptr);
        PGB_CHECK_LAUNCH("k_scatter_f64");
        copy_out(ranks, out.ptr, (size_t)n * 8, mem, s);
        PGB_CUDA(cudaStreamSynchronize(s));
        if (iterations) *iterations = it;
        if (last_change) *last_change = err;
    });
}

}  // extern "C"
