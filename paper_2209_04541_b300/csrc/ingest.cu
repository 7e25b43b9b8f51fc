// Graph ingest (Section 5.1 preprocessing: undirected, duplicates removed,
// self-loops dropped) on the device.
//
// Each raw pair {a, b} becomes its canonical pair (min, max) of B-bit IDs,
// B the bit width of the largest vertex ID; self-loops and invalid IDs
// become (2^B - 1, 2^B - 1), which sorts last.  A lexicographic radix sort
// groups equal pairs, a unique pass keeps one of each as a packed key
// (min << B) | max, and the degree of each vertex is counted from the unique
// pairs.
#include <cub/device/device_merge.cuh>
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_select.cuh>
#include <thrust/iterator/counting_iterator.h>
#include <thrust/iterator/transform_iterator.h>

#include "internal.cuh"
#include "sort.cuh"

namespace pgb {

__global__ void k_canon_pairs(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst, uint64_t m,
                              uint32_t n, uint32_t top, uint32_t* __restrict__ lo, uint32_t* __restrict__ hi,
                              int* __restrict__ err) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        uint32_t a = src[e], b = dst[e];
        uint32_t x = top, y = top;
        if (a >= n || b >= n) {
            atomicOr(err, 1);
        } else if (a != b) {
            x = a < b ? a : b;
            y = a < b ? b : a;
        }
        lo[e] = x;
        hi[e] = y;
    }
}

// Row of CSR entry e: the largest u with offs[u] <= e (offs non-decreasing).
__global__ void k_csr_pairs(const int64_t* __restrict__ offs, const uint32_t* __restrict__ cols, uint32_t n,
                            uint64_t nnz, uint32_t top, uint32_t* __restrict__ lo, uint32_t* __restrict__ hi,
                            int* __restrict__ err) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        uint32_t l = 0, h = n;  // search u in [0, n): offs[u] <= e < offs[u+1]
        while (h - l > 1) {
            uint32_t mid = l + (h - l) / 2;
            if ((uint64_t)offs[mid] <= e) l = mid; else h = mid;
        }
        uint32_t a = l, b = cols[e];
        uint32_t x = top, y = top;
        if (b >= n) {
            atomicOr(err, 1);
        } else if (a != b) {
            x = a < b ? a : b;
            y = a < b ? b : a;
        }
        lo[e] = x;
        hi[e] = y;
    }
}

__global__ void k_check_offs(const int64_t* __restrict__ offs, uint32_t n, int* __restrict__ err) {
    uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride)
        if (offs[u + 1] < offs[u]) atomicOr(err, 2);
    if (blockIdx.x == 0 && threadIdx.x == 0 && offs[0] != 0) atomicOr(err, 2);
}

__global__ void k_degrees(const uint64_t* __restrict__ keys, uint64_t m, uint32_t B, uint32_t* __restrict__ deg) {
    const uint64_t mask = (B >= 64) ? ~0ull : ((1ull << B) - 1);
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        uint64_t k = keys[e];
        const uint32_t a = (uint32_t)(k >> B);
        // keys are sorted, so neighbouring lanes mostly share the first
        // endpoint: one atomic per group of equal endpoints
        const unsigned same = __match_any_sync(__activemask(), a);
        if ((threadIdx.x & 31) == (unsigned)(__ffs(same) - 1)) atomicAdd(&deg[a], (unsigned)__popc(same));
        atomicAdd(&deg[(uint32_t)(k & mask)], 1u);
    }
}

static int grid_for(uint64_t items, int threads = 256) {
    uint64_t g = (items + threads - 1) / threads;
    if (g > 148ull * 32) g = 148ull * 32;
    return g < 1 ? 1 : (int)g;
}

// Packed key (a << B) | b of sorted pair i, read on the fly by the unique pass.
struct PackPair {
    const uint32_t* a;
    const uint32_t* b;
    uint32_t B;
    __host__ __device__ uint64_t operator()(uint64_t i) const { return ((uint64_t)a[i] << B) | b[i]; }
};

// Sort the raw canonical pairs, keep one of each, count degrees.  `lo` and
// `hi` hold the m raw pairs on entry (both are consumed).
static void finish_ingest(pgb_graph* g, DevBuf<uint32_t>& lo, DevBuf<uint32_t>& hi, uint64_t m, DevBuf<int>& err,
                          cudaStream_t s) {
    const uint32_t B = g->id_bits;
    const int end_bit = (int)(2 * B);
    if (m == 0) {
        int herr = 0;
        PGB_CUDA(cudaMemcpyAsync(&herr, err.ptr, sizeof(herr), cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaStreamSynchronize(s));
        if (herr) fail(PGB_E_INVAL, "CSR offsets must start at 0 and be non-decreasing");
        g->m = 0;
        g->deg.alloc(g->n, s);
        if (g->n) PGB_CUDA(cudaMemsetAsync(g->deg.ptr, 0, (size_t)g->n * sizeof(uint32_t), s));
        return;
    }
    Scratch scratch;
    DevBuf<uint64_t> uniq;
    DevBuf<int64_t> nsel(1, s);
    {
        DevBuf<uint32_t> lo_alt(m, s), hi_alt(m, s);
        uint32_t *a, *b;
        sort_pairs_lex(lo.ptr, lo_alt.ptr, hi.ptr, hi_alt.ptr, m, (int)B, s, scratch, &a, &b);
        // free the two scratch halves before the packed output is allocated
        if (a == lo.ptr) lo_alt.release(); else lo.release();
        if (b == hi.ptr) hi_alt.release(); else hi.release();
        uniq.alloc(m, s);
        auto packed = thrust::make_transform_iterator(thrust::make_counting_iterator<uint64_t>(0), PackPair{a, b, B});
        size_t tmp = 0;
        PGB_CUDA(cub::DeviceSelect::Unique(nullptr, tmp, packed, uniq.ptr, nsel.ptr, (int64_t)m, s));
        void* t = scratch.get(tmp, s);
        PGB_CUDA(cub::DeviceSelect::Unique(t, tmp, packed, uniq.ptr, nsel.ptr, (int64_t)m, s));
        // the sorted halves are released here, after the unique pass on s
    }
    int64_t nu = 0;
    int herr = 0;
    PGB_CUDA(cudaMemcpyAsync(&nu, nsel.ptr, sizeof(nu), cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaMemcpyAsync(&herr, err.ptr, sizeof(herr), cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaStreamSynchronize(s));
    if (herr & 1) fail(PGB_E_INVAL, "vertex ID >= n in input");
    if (herr & 2) fail(PGB_E_INVAL, "CSR offsets must start at 0 and be non-decreasing");
    uint64_t mu = (uint64_t)nu;
    if (mu > 0) {
        uint64_t last = 0;
        PGB_CUDA(cudaMemcpyAsync(&last, uniq.ptr + mu - 1, sizeof(last), cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaStreamSynchronize(s));
        const uint64_t sentinel = (end_bit >= 64) ? ~0ull : ((1ull << end_bit) - 1);
        if ((last & sentinel) == sentinel) --mu;
    }
    if (mu >= (1ull << 32)) fail(PGB_E_OVERFLOW, "2^32 or more unique edges are not supported");
    g->m = mu;
    g->deg.alloc(g->n, s);
    if (g->n) PGB_CUDA(cudaMemsetAsync(g->deg.ptr, 0, (size_t)g->n * sizeof(uint32_t), s));
    if (mu) {
        k_degrees<<<grid_for(mu), 256, 0, s>>>(uniq.ptr, mu, B, g->deg.ptr);
        PGB_CHECK_LAUNCH("k_degrees");
    }
    g->keys = std::move(uniq);
}

// ---- host input in chunks
//
// A host edge list is copied in chunks on a second stream; each chunk is
// canonicalised into packed keys (min << B) | max (self-loops and invalid
// pairs become all ones, which sort last) and sorted while the next chunk
// is still on the way, so most of the sorting hides behind the host link.
// The sorted runs are then merged pairwise, and the unique pass and the
// degree count finish the ingest as for device input.
constexpr uint64_t kChunkPairs = 1ull << 25;  // pairs per chunk
constexpr uint64_t kChunkedMin = 1ull << 26;  // host lists of at least this many pairs are chunked

__global__ void k_canon_pack(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst, uint64_t m,
                             uint32_t n, uint32_t B, uint64_t* __restrict__ keys, int* __restrict__ err) {
    const uint64_t sentinel = B >= 32 ? ~0ull : (1ull << (2 * B)) - 1;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const uint32_t a = src[e], b = dst[e];
        uint64_t key = sentinel;
        if (a >= n || b >= n) {
            atomicOr(err, 1);
        } else if (a != b) {
            key = ((uint64_t)(a < b ? a : b) << B) | (a < b ? b : a);
        }
        keys[e] = key;
    }
}

// Sorted packed keys of the m host pairs, in `out` (m entries); `spare` is
// an m-entry scratch buffer.
static void sort_host_chunked(const pgb_graph* g, const uint32_t* src, const uint32_t* dst, uint64_t m,
                              DevBuf<uint64_t>& out, DevBuf<uint64_t>& spare, const DevBuf<int>& err,
                              cudaStream_t s) {
    const uint32_t B = g->id_bits;
    const int end_bit = (int)(2 * B);
    const uint64_t C = kChunkPairs;
    Scratch scratch;
    DevBuf<uint32_t> stage(4 * C, s);  // two (src, dst) staging pairs
    cudaStream_t cs = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr}, used[2] = {nullptr, nullptr};
    auto cleanup = [&] {
        for (cudaEvent_t e : copied)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : used)
            if (e) cudaEventDestroy(e);
        if (cs) cudaStreamDestroy(cs);
    };
    try {
        PGB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        for (int k = 0; k < 2; ++k) {
            PGB_CUDA(cudaEventCreateWithFlags(&copied[k], cudaEventDisableTiming));
            PGB_CUDA(cudaEventCreateWithFlags(&used[k], cudaEventDisableTiming));
            // the staging memory was allocated on s: the copy stream starts after that
            PGB_CUDA(cudaEventRecord(used[k], s));
        }
        size_t sort_tmp = 0;
        {
            cub::DoubleBuffer<uint64_t> db(out.ptr, spare.ptr);
            PGB_CUDA(cub::DeviceRadixSort::SortKeys(nullptr, sort_tmp, db, (int64_t)C, 0, end_bit, s));
        }
        void* tmp = scratch.get(sort_tmp, s);
        uint64_t i = 0;
        for (uint64_t off = 0; off < m; off += C, ++i) {
            const int k = (int)(i & 1);
            const uint64_t len = m - off < C ? m - off : C;
            uint32_t* cs_src = stage.ptr + (size_t)k * 2 * C;
            uint32_t* cs_dst = cs_src + C;
            PGB_CUDA(cudaStreamWaitEvent(cs, used[k], 0));
            PGB_CUDA(cudaMemcpyAsync(cs_src, src + off, len * 4, cudaMemcpyHostToDevice, cs));
            PGB_CUDA(cudaMemcpyAsync(cs_dst, dst + off, len * 4, cudaMemcpyHostToDevice, cs));
            PGB_CUDA(cudaEventRecord(copied[k], cs));
            PGB_CUDA(cudaStreamWaitEvent(s, copied[k], 0));
            k_canon_pack<<<grid_for(len), 256, 0, s>>>(cs_src, cs_dst, len, g->n, B, out.ptr + off, err.ptr);
            PGB_CHECK_LAUNCH("k_canon_pack");
            PGB_CUDA(cudaEventRecord(used[k], s));
            cub::DoubleBuffer<uint64_t> db(out.ptr + off, spare.ptr + off);
            size_t t = sort_tmp;
            PGB_CUDA(cub::DeviceRadixSort::SortKeys(tmp, t, db, (int64_t)len, 0, end_bit, s));
            if (db.Current() != out.ptr + off)
                PGB_CUDA(cudaMemcpyAsync(out.ptr + off, db.Current(), len * 8, cudaMemcpyDeviceToDevice, s));
        }
    } catch (...) {
        cudaStreamSynchronize(s);
        if (cs) cudaStreamSynchronize(cs);
        cleanup();
        throw;
    }
    cleanup();
    // merge the sorted runs pairwise until one run is left; `out` ends up
    // holding the result
    for (uint64_t run = C; run < m; run *= 2) {
        for (uint64_t a0 = 0; a0 < m; a0 += 2 * run) {
            const uint64_t a1 = a0 + run < m ? a0 + run : m, b1 = a0 + 2 * run < m ? a0 + 2 * run : m;
            if (a1 == b1) {  // no partner in this round: carried over
                PGB_CUDA(cudaMemcpyAsync(spare.ptr + a0, out.ptr + a0, (a1 - a0) * 8, cudaMemcpyDeviceToDevice, s));
                continue;
            }
            size_t t = 0;
            PGB_CUDA(cub::DeviceMerge::MergeKeys(nullptr, t, out.ptr + a0, (int64_t)(a1 - a0), out.ptr + a1,
                                                 (int64_t)(b1 - a1), spare.ptr + a0, ::cuda::std::less<>{}, s));
            void* tm = scratch.get(t, s);
            PGB_CUDA(cub::DeviceMerge::MergeKeys(tm, t, out.ptr + a0, (int64_t)(a1 - a0), out.ptr + a1,
                                                 (int64_t)(b1 - a1), spare.ptr + a0, ::cuda::std::less<>{}, s));
        }
        out.swap(spare);
    }
}

// Unique pass and degree count over sorted packed keys (`sorted`, m
// entries); `spare` (m entries) receives the unique keys and becomes the
// graph's.  Fails on the error flags first.
static void finish_sorted(pgb_graph* g, DevBuf<uint64_t>& sorted, DevBuf<uint64_t>& spare, uint64_t m,
                          const DevBuf<int>& err, cudaStream_t s) {
    const uint32_t B = g->id_bits;
    const int end_bit = (int)(2 * B);
    Scratch scratch;
    DevBuf<int64_t> nsel(1, s);
    size_t tmp = 0;
    PGB_CUDA(cub::DeviceSelect::Unique(nullptr, tmp, sorted.ptr, spare.ptr, nsel.ptr, (int64_t)m, s));
    void* t = scratch.get(tmp, s);
    PGB_CUDA(cub::DeviceSelect::Unique(t, tmp, sorted.ptr, spare.ptr, nsel.ptr, (int64_t)m, s));
    sorted.release();
    int64_t nu = 0;
    int herr = 0;
    PGB_CUDA(cudaMemcpyAsync(&nu, nsel.ptr, sizeof(nu), cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaMemcpyAsync(&herr, err.ptr, sizeof(herr), cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaStreamSynchronize(s));
    if (herr & 1) fail(PGB_E_INVAL, "vertex ID >= n in input");
    uint64_t mu = (uint64_t)nu;
    if (mu > 0) {
        uint64_t last = 0;
        PGB_CUDA(cudaMemcpyAsync(&last, spare.ptr + mu - 1, sizeof(last), cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaStreamSynchronize(s));
        const uint64_t sentinel = (end_bit >= 64) ? ~0ull : ((1ull << end_bit) - 1);
        if ((last & sentinel) == sentinel) --mu;
    }
    if (mu >= (1ull << 32)) fail(PGB_E_OVERFLOW, "2^32 or more unique edges are not supported");
    g->m = mu;
    g->deg.alloc(g->n, s);
    if (g->n) PGB_CUDA(cudaMemsetAsync(g->deg.ptr, 0, (size_t)g->n * sizeof(uint32_t), s));
    if (mu) {
        k_degrees<<<grid_for(mu), 256, 0, s>>>(spare.ptr, mu, B, g->deg.ptr);
        PGB_CHECK_LAUNCH("k_degrees");
    }
    g->keys = std::move(spare);
}
static pgb_graph* new_graph(uint32_t n, cudaStream_t s) {
    pgb_graph* g = new pgb_graph();
    g->n = n;
    g->stream = s;
    g->id_bits = (uint32_t)num_bits(n > 0 ? (uint64_t)n - 1 : 0);
    return g;
}

}  // namespace pgb

using namespace pgb;

extern "C" {

int pgb_graph_from_edges(const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n, int mem,
                         void* stream, pgb_graph** out) {
    return guard([&] {
        if (!out) fail(PGB_E_INVAL, "out is NULL");
        if (m > 0 && (!src || !dst)) fail(PGB_E_INVAL, "src/dst NULL with m > 0");
        if (mem != PGB_MEM_HOST && mem != PGB_MEM_DEVICE) fail(PGB_E_INVAL, "bad mem kind");
        if (m > 0 && n == 0) fail(PGB_E_INVAL, "edges given for an empty vertex set");
        cudaStream_t s = (cudaStream_t)stream;
        std::unique_ptr<pgb_graph> g(new_graph(n, s));
        const uint32_t top = (uint32_t)((1ull << g->id_bits) - 1);  // the (top, top) pair sorts last
        if (mem == PGB_MEM_HOST && m >= kChunkedMin) {
            // host input: sorted per chunk behind the copies, then merged
            DevBuf<int> err(1, s);
            PGB_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
            DevBuf<uint64_t> keys(m, s), spare(m, s);
            sort_host_chunked(g.get(), src, dst, m, keys, spare, err, s);
            finish_sorted(g.get(), keys, spare, m, err, s);
            live_handles_add(1);
            *out = g.release();
            return;
        }
        DevBuf<uint32_t> lo(m, s), hi(m, s);
        DevBuf<int> err(1, s);
        PGB_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
        if (m > 0) {
            const uint32_t* ds = src;
            const uint32_t* dd = dst;
            DevBuf<uint32_t> hs, hd;
            if (mem == PGB_MEM_HOST) {
                hs.alloc(m, s);
                hd.alloc(m, s);
                PGB_CUDA(cudaMemcpyAsync(hs.ptr, src, m * 4, cudaMemcpyHostToDevice, s));
                PGB_CUDA(cudaMemcpyAsync(hd.ptr, dst, m * 4, cudaMemcpyHostToDevice, s));
                ds = hs.ptr;
                dd = hd.ptr;
            }
            k_canon_pairs<<<grid_for(m), 256, 0, s>>>(ds, dd, m, n, top, lo.ptr, hi.ptr, err.ptr);
            PGB_CHECK_LAUNCH("k_canon_pairs");
        }
        finish_ingest(g.get(), lo, hi, m, err, s);
        live_handles_add(1);
        *out = g.release();
    });
}

int pgb_graph_from_csr(uint32_t n, const int64_t* offs, const uint32_t* cols, int mem, void* stream,
                       pgb_graph** out) {
    return guard([&] {
        if (!out || !offs) fail(PGB_E_INVAL, "NULL argument");
        if (mem != PGB_MEM_HOST && mem != PGB_MEM_DEVICE) fail(PGB_E_INVAL, "bad mem kind");
        cudaStream_t s = (cudaStream_t)stream;
        std::unique_ptr<pgb_graph> g(new_graph(n, s));
        const uint32_t top = (uint32_t)((1ull << g->id_bits) - 1);  // the (top, top) pair sorts last
        DevBuf<int64_t> hoffs;
        const int64_t* doffs = offs;
        int64_t nnz = 0;
        if (mem == PGB_MEM_HOST) {
            nnz = offs[n];
            hoffs.alloc((size_t)n + 1, s);
            PGB_CUDA(cudaMemcpyAsync(hoffs.ptr, offs, ((size_t)n + 1) * 8, cudaMemcpyHostToDevice, s));
            doffs = hoffs.ptr;
        } else {
            PGB_CUDA(cudaMemcpyAsync(&nnz, offs + n, 8, cudaMemcpyDeviceToHost, s));
            PGB_CUDA(cudaStreamSynchronize(s));
        }
        if (nnz < 0) fail(PGB_E_INVAL, "negative CSR size");
        if (nnz > 0 && !cols) fail(PGB_E_INVAL, "cols NULL with entries");
        DevBuf<int> err(1, s);
        PGB_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
        if (n > 0) {
            k_check_offs<<<grid_for(n), 256, 0, s>>>(doffs, n, err.ptr);
            PGB_CHECK_LAUNCH("k_check_offs");
        }
        int herr = 0;
        PGB_CUDA(cudaMemcpyAsync(&herr, err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaStreamSynchronize(s));
        if (herr) fail(PGB_E_INVAL, "CSR offsets must start at 0 and be non-decreasing");
        DevBuf<uint32_t> lo((size_t)nnz, s), hi((size_t)nnz, s);
        if (nnz > 0) {
            const uint32_t* dcols = cols;
            DevBuf<uint32_t> hcols;
            if (mem == PGB_MEM_HOST) {
                hcols.alloc((size_t)nnz, s);
                PGB_CUDA(cudaMemcpyAsync(hcols.ptr, cols, (size_t)nnz * 4, cudaMemcpyHostToDevice, s));
                dcols = hcols.ptr;
            }
            k_csr_pairs<<<grid_for(nnz), 256, 0, s>>>(doffs, dcols, n, (uint64_t)nnz, top, lo.ptr, hi.ptr, err.ptr);
            PGB_CHECK_LAUNCH("k_csr_pairs");
        }
        finish_ingest(g.get(), lo, hi, (uint64_t)nnz, err, s);
        live_handles_add(1);
        *out = g.release();
    });
}

int pgb_graph_info(const pgb_graph* g, uint32_t* n, uint64_t* m_undirected) {
    return guard([&] {
        if (!g) fail(PGB_E_INVAL, "graph is NULL");
        if (n) *n = g->n;
        if (m_undirected) *m_undirected = g->m;
    });
}

__global__ void k_unpack_keys(const uint64_t* __restrict__ keys, uint64_t m, uint32_t B, uint32_t* a, uint32_t* b) {
    const uint64_t mask = (B >= 64) ? ~0ull : ((1ull << B) - 1);
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        uint64_t k = keys[e];
        if (a) a[e] = (uint32_t)(k >> B);
        if (b) b[e] = (uint32_t)(k & mask);
    }
}

int pgb_graph_export(const pgb_graph* g, uint32_t* a, uint32_t* b, uint32_t* deg, int mem, void* stream) {
    return guard([&] {
        if (!g) fail(PGB_E_INVAL, "graph is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        if ((a || b) && g->m) {
            DevBuf<uint32_t> da(g->m, s), db(g->m, s);
            k_unpack_keys<<<grid_for(g->m), 256, 0, s>>>(g->keys.ptr, g->m, g->id_bits, da.ptr, db.ptr);
            PGB_CHECK_LAUNCH("k_unpack_keys");
            if (a) copy_out(a, da.ptr, g->m * 4, mem, s);
            if (b) copy_out(b, db.ptr, g->m * 4, mem, s);
            PGB_CUDA(cudaStreamSynchronize(s));
        }
        if (deg && g->n) copy_out(deg, g->deg.ptr, (size_t)g->n * 4, mem, s);
    });
}

void pgb_graph_free(pgb_graph* g) {
    if (!g) return;
    delete g;
    live_handles_add(-1);
}

}  // extern "C"
