// Graph ingest (Section 5.1 preprocessing: undirected, duplicates removed,
// self-loops dropped) on the device.
//
// Each raw pair {a, b} becomes one canonical key (min << B) | max, where B
// is the bit width of the largest vertex ID; self-loops and invalid IDs
// become an all-ones sentinel that sorts last.  One radix sort over the 2B
// significant bits groups equal pairs, a unique pass keeps one of each, and
// the degree of each vertex is counted from the unique pairs.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_select.cuh>

#include "internal.cuh"

namespace pgb {

__global__ void k_canon_keys(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst, uint64_t m,
                             uint32_t n, uint32_t B, uint64_t sentinel, uint64_t* __restrict__ keys,
                             int* __restrict__ err) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        uint32_t a = src[e], b = dst[e];
        uint64_t k = sentinel;
        if (a >= n || b >= n) {
            atomicOr(err, 1);
        } else if (a != b) {
            uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
            k = ((uint64_t)lo << B) | hi;
        }
        keys[e] = k;
    }
}

// Row of CSR entry e: the largest u with offs[u] <= e (offs non-decreasing).
__global__ void k_csr_keys(const int64_t* __restrict__ offs, const uint32_t* __restrict__ cols, uint32_t n,
                           uint64_t nnz, uint32_t B, uint64_t sentinel, uint64_t* __restrict__ keys,
                           int* __restrict__ err) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        uint32_t lo = 0, hi = n;  // search u in [0, n): offs[u] <= e < offs[u+1]
        while (hi - lo > 1) {
            uint32_t mid = lo + (hi - lo) / 2;
            if ((uint64_t)offs[mid] <= e) lo = mid; else hi = mid;
        }
        uint32_t a = lo, b = cols[e];
        uint64_t k = sentinel;
        if (b >= n) {
            atomicOr(err, 1);
        } else if (a != b) {
            uint32_t x = a < b ? a : b, y = a < b ? b : a;
            k = ((uint64_t)x << B) | y;
        }
        keys[e] = k;
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

// Sort the raw keys, keep one of each, count degrees.  `keys` holds m raw
// keys on entry; the graph takes ownership of the buffer with the result.
static void finish_ingest(pgb_graph* g, DevBuf<uint64_t>& keys, uint64_t m, DevBuf<int>& err, cudaStream_t s) {
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
    DevBuf<uint64_t> alt(m, s);
    Scratch scratch;
    cub::DoubleBuffer<uint64_t> db(keys.ptr, alt.ptr);
    size_t tmp = 0;
    PGB_CUDA(cub::DeviceRadixSort::SortKeys(nullptr, tmp, db, (int64_t)m, 0, end_bit, s));
    void* t = scratch.get(tmp, s);
    PGB_CUDA(cub::DeviceRadixSort::SortKeys(t, tmp, db, (int64_t)m, 0, end_bit, s));
    uint64_t* sorted = db.Current();
    uint64_t* uniq = (sorted == keys.ptr) ? alt.ptr : keys.ptr;
    DevBuf<int64_t> nsel(1, s);
    size_t tmp2 = 0;
    PGB_CUDA(cub::DeviceSelect::Unique(nullptr, tmp2, sorted, uniq, nsel.ptr, (int64_t)m, s));
    t = scratch.get(tmp2, s);
    PGB_CUDA(cub::DeviceSelect::Unique(t, tmp2, sorted, uniq, nsel.ptr, (int64_t)m, s));
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
        PGB_CUDA(cudaMemcpyAsync(&last, uniq + mu - 1, sizeof(last), cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaStreamSynchronize(s));
        const uint64_t sentinel = (end_bit >= 64) ? ~0ull : ((1ull << end_bit) - 1);
        if ((last & sentinel) == sentinel) --mu;
    }
    if (mu >= (1ull << 32)) fail(PGB_E_OVERFLOW, "2^32 or more unique edges are not supported");
    g->m = mu;
    g->deg.alloc(g->n, s);
    if (g->n) PGB_CUDA(cudaMemsetAsync(g->deg.ptr, 0, (size_t)g->n * sizeof(uint32_t), s));
    if (mu) {
        k_degrees<<<grid_for(mu), 256, 0, s>>>(uniq, mu, B, g->deg.ptr);
        PGB_CHECK_LAUNCH("k_degrees");
    }
    if (uniq == keys.ptr) {
        g->keys = std::move(keys);
    } else {
        g->keys = std::move(alt);
    }
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
        const uint32_t B = g->id_bits;
        const uint64_t sentinel = (2 * B >= 64) ? ~0ull : ((1ull << (2 * B)) - 1);
        DevBuf<uint64_t> keys(m, s);
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
            k_canon_keys<<<grid_for(m), 256, 0, s>>>(ds, dd, m, n, B, sentinel, keys.ptr, err.ptr);
            PGB_CHECK_LAUNCH("k_canon_keys");
        }
        finish_ingest(g.get(), keys, m, err, s);
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
        const uint32_t B = g->id_bits;
        const uint64_t sentinel = (2 * B >= 64) ? ~0ull : ((1ull << (2 * B)) - 1);
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
        DevBuf<uint64_t> keys((size_t)nnz, s);
        if (nnz > 0) {
            const uint32_t* dcols = cols;
            DevBuf<uint32_t> hcols;
            if (mem == PGB_MEM_HOST) {
                hcols.alloc((size_t)nnz, s);
                PGB_CUDA(cudaMemcpyAsync(hcols.ptr, cols, (size_t)nnz * 4, cudaMemcpyHostToDevice, s));
                dcols = hcols.ptr;
            }
            k_csr_keys<<<grid_for(nnz), 256, 0, s>>>(doffs, dcols, n, (uint64_t)nnz, B, sentinel, keys.ptr, err.ptr);
            PGB_CHECK_LAUNCH("k_csr_keys");
        }
        finish_ingest(g.get(), keys, (uint64_t)nnz, err, s);
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
