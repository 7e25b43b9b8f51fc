// Block layout and block storage formats (PGAbB Section 4.3.1 and 4.3.2).
//
// Layout: every block gets an integer ID; the default order is row-major,
// and Section 4.3.1 allows any space-filling curve instead.  pgb_block_order
// lists the upper blocks (i <= j) in row-major or Hilbert-curve order; the
// Hilbert order is also a queue order for plain (per-triple) runs, where
// consecutive launches then share blocks.
//
// Storage: inside the library a block A_ij is an implicit slice of the
// oriented CSR (rows of V_i, columns clipped to V_j), so the counting kernels
// need no second copy of the graph.  For callers, any block can be
// materialised with block-local vertex IDs (u - c_i, v - c_j) in one of the
// three formats of Section 4.3.2: CSR (offsets over all rows of the block),
// COO (one (row, column) pair per edge) and CCOO (compact: offsets over the
// non-empty rows only, with their row IDs).  The format chosen per block is
// the one with the fewest bytes for that block's shape: CCOO for blocks
// whose rows are mostly empty, COO for about one edge per non-empty row,
// CSR otherwise.
//
// Hilbert index of cell (x, y) in a 2^k x 2^k grid: the standard
// quadrant-by-quadrant construction (each level adds the quadrant's offset
// along the curve, then rotates or flips the coordinates so that the
// sub-curve inside the quadrant has the same orientation).
#include <cub/device/device_scan.cuh>

#include <algorithm>

#include "internal.cuh"

namespace pgb {

namespace {

uint64_t hilbert_index(uint32_t side_pow2, uint32_t x, uint32_t y) {
    uint64_t d = 0;
    for (uint32_t s = side_pow2 / 2; s > 0; s /= 2) {
        const uint32_t rx = (x & s) ? 1u : 0u, ry = (y & s) ? 1u : 0u;
        d += (uint64_t)s * s * ((3u * rx) ^ ry);
        if (ry == 0) {  // rotate the quadrant
            if (rx == 1) {
                x = s - 1 - (x & (s - 1));
                y = s - 1 - (y & (s - 1));
            }
            std::swap(x, y);
        }
        x &= s - 1;
        y &= s - 1;
    }
    return d;
}

uint32_t pow2_at_least(uint32_t p) {
    uint32_t s = 1;
    while (s < p) s <<= 1;
    return s;
}

// Per row u of V_i: the slice of its columns inside [lo, hi).
__global__ void k_block_slices(const uint32_t* __restrict__ rowptr, const uint32_t* __restrict__ col, uint32_t r0,
                               uint32_t rows, uint32_t lo, uint32_t hi, uint32_t* __restrict__ start,
                               uint32_t* __restrict__ len, uint32_t* __restrict__ nonempty) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < rows; k += stride) {
        const uint32_t u = r0 + k;
        uint32_t b = rowptr[u], e = rowptr[u + 1];
        uint32_t a = b, z = e;
        while (a < z) {  // first entry >= lo
            const uint32_t mid = a + ((z - a) >> 1);
            if (col[mid] < lo) a = mid + 1; else z = mid;
        }
        uint32_t c = a;
        z = e;
        while (c < z) {  // first entry >= hi
            const uint32_t mid = c + ((z - c) >> 1);
            if (col[mid] < hi) c = mid + 1; else z = mid;
        }
        start[k] = a;
        len[k] = c - a;
        nonempty[k] = c > a ? 1u : 0u;
    }
}

// Writes the block in the requested format from the per-row slices and
// their exclusive scans (off: edges before row k; nzoff: non-empty rows
// before row k).
__global__ void k_block_write(const uint32_t* __restrict__ col, uint32_t rows, uint32_t cbase,
                              const uint32_t* __restrict__ start, const uint32_t* __restrict__ len,
                              const uint32_t* __restrict__ off, const uint32_t* __restrict__ nzoff, int format,
                              uint32_t* __restrict__ a, uint32_t* __restrict__ c, uint32_t* __restrict__ d) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < rows; k += stride) {
        const uint32_t o = off[k], l = len[k], s = start[k];
        for (uint32_t t = 0; t < l; ++t) {
            c[o + t] = col[s + t] - cbase;
            if (format == PGB_FMT_COO) a[o + t] = k;
        }
        if (format == PGB_FMT_CSR) {
            a[k] = o;
            if (k + 1 == rows) a[rows] = o + l;
        } else if (format == PGB_FMT_CCOO && l) {
            a[nzoff[k]] = k;
            d[nzoff[k]] = o;
        }
    }
}

struct BlockShape {
    uint32_t rows, cols, nonempty;
    uint64_t nnz;
};

// Per-row slices of block (i, j) on the device; nonempty rows counted.
BlockShape block_shape(const pgb_blocks* b, uint32_t i, uint32_t j, cudaStream_t s, DevBuf<uint32_t>& start,
                       DevBuf<uint32_t>& len, DevBuf<uint32_t>& nz, DevBuf<uint32_t>& off, DevBuf<uint32_t>& nzoff) {
    BlockShape z;
    const uint32_t r0 = b->cuts[i];
    z.rows = b->cuts[i + 1] - r0;
    z.cols = b->cuts[j + 1] - b->cuts[j];
    z.nnz = b->block_edges[(size_t)i * b->p + j];
    z.nonempty = 0;
    if (z.rows == 0) return z;
    start.alloc(z.rows, s);
    len.alloc(z.rows, s);
    nz.alloc(z.rows + 1, s);
    off.alloc(z.rows + 1, s);
    nzoff.alloc(z.rows + 1, s);
    PGB_CUDA(cudaMemsetAsync(nz.ptr + z.rows, 0, 4, s));
    const unsigned grid = (unsigned)std::min<uint64_t>((z.rows + 255) / 256, 148ull * 16);
    k_block_slices<<<grid, 256, 0, s>>>(b->rowptr.ptr, b->col.ptr, r0, z.rows, b->cuts[j], b->cuts[j + 1], start.ptr,
                                        len.ptr, nz.ptr);
    PGB_CHECK_LAUNCH("k_block_slices");
    Scratch scratch;
    size_t t1 = 0, t2 = 0;
    PGB_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, t1, len.ptr, off.ptr, (int)z.rows, s));
    PGB_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, t2, nz.ptr, nzoff.ptr, (int)z.rows + 1, s));
    void* t = scratch.get(std::max(t1, t2), s);
    PGB_CUDA(cub::DeviceScan::ExclusiveSum(t, t1, len.ptr, off.ptr, (int)z.rows, s));
    PGB_CUDA(cub::DeviceScan::ExclusiveSum(t, t2, nz.ptr, nzoff.ptr, (int)z.rows + 1, s));
    PGB_CUDA(cudaMemcpyAsync(&z.nonempty, nzoff.ptr + z.rows, 4, cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaStreamSynchronize(s));
    return z;
}

// Bytes of each format for a block of this shape.
uint64_t format_bytes(int f, const BlockShape& z) {
    if (f == PGB_FMT_CSR) return 4ull * ((uint64_t)z.rows + 1 + z.nnz);
    if (f == PGB_FMT_COO) return 8ull * z.nnz;
    return 4ull * (2ull * z.nonempty + 1 + z.nnz);
}

int best_format(const BlockShape& z) {
    int best = PGB_FMT_CSR;
    for (int f : {PGB_FMT_COO, PGB_FMT_CCOO})
        if (format_bytes(f, z) < format_bytes(best, z)) best = f;
    return best;
}

void check_block(const pgb_blocks* b, uint32_t i, uint32_t j) {
    if (!b) fail(PGB_E_INVAL, "blocks is NULL");
    if (i >= b->p || j >= b->p) fail(PGB_E_INVAL, "block index out of range");
    if (b->cols_offloaded) fail(PGB_E_STATE, "the columns are offloaded");
}

}  // namespace

std::vector<uint32_t> hilbert_block_order(uint32_t p) {
    std::vector<std::pair<uint64_t, uint32_t>> key;
    const uint32_t side = pow2_at_least(p);
    for (uint32_t i = 0; i < p; ++i)
        for (uint32_t j = i; j < p; ++j) key.emplace_back(hilbert_index(side, j, i), i * p + j);
    std::sort(key.begin(), key.end());
    std::vector<uint32_t> ids;
    for (auto& k : key) ids.push_back(k.second);
    return ids;
}

}  // namespace pgb

using namespace pgb;

extern "C" {

int pgb_hilbert_index(uint32_t side, uint32_t x, uint32_t y, uint64_t* d) {
    return guard([&] {
        if (!d) fail(PGB_E_INVAL, "d is NULL");
        if (side == 0 || (side & (side - 1))) fail(PGB_E_INVAL, "side must be a power of two");
        if (x >= side || y >= side) fail(PGB_E_INVAL, "cell outside the grid");
        *d = hilbert_index(side, x, y);
    });
}

int pgb_block_order(uint32_t p, int layout, uint32_t* ij) {
    return guard([&] {
        if (!ij) fail(PGB_E_INVAL, "ij is NULL");
        if (p == 0 || p > 1024) fail(PGB_E_INVAL, "p must be in [1, 1024]");
        if (layout != PGB_LAYOUT_ROWMAJOR && layout != PGB_LAYOUT_HILBERT) fail(PGB_E_INVAL, "bad block layout");
        std::vector<uint32_t> ids;
        if (layout == PGB_LAYOUT_HILBERT) {
            ids = hilbert_block_order(p);
        } else {
            for (uint32_t i = 0; i < p; ++i)
                for (uint32_t j = i; j < p; ++j) ids.push_back(i * p + j);
        }
        for (size_t t = 0; t < ids.size(); ++t) {
            ij[2 * t] = ids[t] / p;
            ij[2 * t + 1] = ids[t] % p;
        }
    });
}

int pgb_blocks_block_info(const pgb_blocks* b, uint32_t i, uint32_t j, pgb_block_info* out) {
    return guard([&] {
        check_block(b, i, j);
        if (!out) fail(PGB_E_INVAL, "out is NULL");
        cudaStream_t s = b->stream;
        DevBuf<uint32_t> start, len, nz, off, nzoff;
        const BlockShape z = block_shape(b, i, j, s, start, len, nz, off, nzoff);
        std::memset(out, 0, sizeof(*out));
        out->rows = z.rows;
        out->cols = z.cols;
        out->nnz = z.nnz;
        out->nonempty_rows = z.nonempty;
        out->format = best_format(z);
        out->bytes_csr = format_bytes(PGB_FMT_CSR, z);
        out->bytes_coo = format_bytes(PGB_FMT_COO, z);
        out->bytes_ccoo = format_bytes(PGB_FMT_CCOO, z);
    });
}

int pgb_blocks_export_block(const pgb_blocks* b, uint32_t i, uint32_t j, int format, uint32_t* a, uint32_t* c,
                            uint32_t* d, int mem, void* stream) {
    return guard([&] {
        check_block(b, i, j);
        if (format != PGB_FMT_CSR && format != PGB_FMT_COO && format != PGB_FMT_CCOO) fail(PGB_E_INVAL, "bad format");
        cudaStream_t s = (cudaStream_t)stream;
        DevBuf<uint32_t> start, len, nz, off, nzoff;
        const BlockShape z = block_shape(b, i, j, s, start, len, nz, off, nzoff);
        const uint64_t na = format == PGB_FMT_CSR ? (uint64_t)z.rows + 1 : format == PGB_FMT_COO ? z.nnz : z.nonempty;
        if ((na && !a) || (z.nnz && !c) || (format == PGB_FMT_CCOO && !d))
            fail(PGB_E_INVAL, "NULL output array for a non-empty block");
        DevBuf<uint32_t> da(std::max<uint64_t>(na, 1), s), dc(std::max<uint64_t>(z.nnz, 1), s),
            dd((uint64_t)z.nonempty + 1, s);
        if (z.rows == 0) {
            if (format == PGB_FMT_CSR) PGB_CUDA(cudaMemsetAsync(da.ptr, 0, 4, s));
        } else {
            const unsigned grid = (unsigned)std::min<uint64_t>((z.rows + 255) / 256, 148ull * 16);
            k_block_write<<<grid, 256, 0, s>>>(b->col.ptr, z.rows, b->cuts[j], start.ptr, len.ptr, off.ptr, nzoff.ptr,
                                               format, da.ptr, dc.ptr, dd.ptr);
            PGB_CHECK_LAUNCH("k_block_write");
        }
        if (format == PGB_FMT_CCOO) {
            const uint32_t nnz32 = (uint32_t)z.nnz;
            PGB_CUDA(cudaMemcpyAsync(dd.ptr + z.nonempty, &nnz32, 4, cudaMemcpyHostToDevice, s));
            copy_out(d, dd.ptr, ((size_t)z.nonempty + 1) * 4, mem, s);
        }
        copy_out(a, da.ptr, na * 4, mem, s);
        copy_out(c, dc.ptr, z.nnz * 4, mem, s);
        PGB_CUDA(cudaStreamSynchronize(s));
    });
}

}  // extern "C"
