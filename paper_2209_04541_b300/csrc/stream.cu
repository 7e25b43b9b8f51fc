// Streaming tier: triangle counting when the in-edge index lives in pinned
// host memory (PGAbB Section 4.4: the scheduler copies a task's blocks to
// the device asynchronously; Section 1: graphs that fit in host DRAM but not
// in device memory).
//
// After pgb_blocks_offload the device keeps what the counting kernel reads
// at random (row offsets, columns, in-edge offsets, the rank permutation);
// the in-edge index -- for every in-edge, grouped by head, the range of the
// tail's row after the head (8 bytes) and the tail (4 bytes) -- moves to
// pinned host memory.  A run cuts the work items, in in-edge order, into
// chunks whose in-edges fit one of two device slots of device_budget / 2
// bytes, and overlaps the copy of chunk c + 1 (side stream) with the
// counting launch of chunk c (run stream).
#include <algorithm>
#include <cub/cub.cuh>

#include "internal.cuh"
#include "tc_hash.cuh"

namespace pgb {

__global__ void k_gather_tails(const unsigned long long* __restrict__ xr, uint64_t m,
                               const uint32_t* __restrict__ rowidx, uint32_t* __restrict__ itail) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
        itail[i] = rowidx[(uint32_t)xr[i] - 1];
}

static int grid_for(uint64_t items) {
    uint64_t g = (items + 255) / 256;
    if (g > 148ull * 32) g = 148ull * 32;
    return g < 1 ? 1 : (int)g;
}

// Bytes per streamed in-edge: the tail-row range (8) and the tail (4).
constexpr uint64_t kStreamBytesPerInEdge = 12;
// Partials of all launches of one run: grid totals per chunk (the chunk
// count is capped so that they fit).
constexpr uint64_t kPartialsReserve = 16ull << 20;
// Slot size when no budget is given.
constexpr uint64_t kDefaultSlotBytes = 1ull << 30;

// Device bytes a streamed run holds besides its two slots.
static uint64_t resident_bytes(const pgb_blocks* b, bool pv) {
    const uint64_t n = b->n;
    return 4 * (n + 1) + 4 * (b->m + 8) + 4 * (n + 1) + 4 * n + 4 * ((uint64_t)b->p + 1) + (pv ? 16 * n : 0) +
           kPartialsReserve;
}

// The chunking of one (work-item size, budget, per-vertex) setting, kept on
// the blocks handle: building it needs the items on the host once.
struct StreamPlan {
    struct Chunk {
        uint32_t first, count, base, span;  // items [first, first+count), in-edges [base, base+span)
    };
    uint32_t in_chunk = 0;
    uint64_t budget = 0;
    bool pv = false;
    uint32_t threads_opt = 0;
    int grid = 0, threads = 128;
    std::vector<Chunk> chunks;
    VItem* h_items = nullptr;  // pinned, in-edge ranges relative to their chunk's base
    uint32_t nitems = 0, max_items = 0;
    uint64_t slot_edges = 0;
    ~StreamPlan() {
        if (h_items) cudaFreeHost(h_items);
    }
};

static std::shared_ptr<StreamPlan> make_plan(const pgb_blocks* b, uint32_t in_chunk, bool pv, uint32_t threads,
                                             uint64_t budget, cudaStream_t s) {
    auto P = std::make_shared<StreamPlan>();
    P->in_chunk = in_chunk;
    P->budget = budget;
    P->pv = pv;
    P->threads_opt = threads;
    P->threads = threads ? (int)threads : hash_threads(b->n);
    P->grid = hash_grid(pv, P->threads);
    // the budget covers everything the run holds on the device: the resident
    // arrays, the per-vertex counters, the per-launch partials (bounded by
    // kPartialsReserve) and the two stream slots
    const uint64_t resident = resident_bytes(b, pv);
    uint64_t slot_bytes = kDefaultSlotBytes;
    if (budget) {
        if (budget <= resident)
            fail(PGB_E_BUDGET, "device_budget of " + std::to_string(budget) + " bytes is below the " +
                                   std::to_string(resident) + " bytes the resident arrays need");
        slot_bytes = (budget - resident) / 2;
    }
    const uint64_t cap = slot_bytes / (kStreamBytesPerInEdge + sizeof(VItem));  // in-edges per slot
    DevBuf<VItem> ditems;
    const uint32_t nitems = build_hash_items(b, in_chunk, P->threads, s, ditems);
    P->nitems = nitems;
    if (nitems == 0) return P;
    std::vector<VItem> items(nitems);
    PGB_CUDA(cudaMemcpyAsync(items.data(), ditems.ptr, (size_t)nitems * sizeof(VItem), cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaStreamSynchronize(s));
    ditems.release();
    // work items in in-edge order; a chunk is a run of items whose in-edge
    // span fits one slot
    if (!std::is_sorted(items.begin(), items.end(),
                        [](const VItem& x, const VItem& y) { return x.in_begin < y.in_begin; }))
        std::stable_sort(items.begin(), items.end(),
                         [](const VItem& x, const VItem& y) { return x.in_begin < y.in_begin; });
    for (uint32_t i = 0; i < nitems;) {
        StreamPlan::Chunk c{i, 0, items[i].in_begin, 0};
        uint32_t end = items[i].in_end;
        // a slot holds the chunk's in-edges and its items; sizing both by
        // the larger of the two counts keeps the two slot arrays fixed
        auto fits = [&](uint32_t e, uint32_t cnt) { return std::max<uint64_t>(e - c.base, cnt) <= cap; };
        if (!fits(end, 1))
            fail(PGB_E_BUDGET, "device_budget too small: one work item needs " +
                                   std::to_string(2 * (uint64_t)(end - c.base) *
                                                  (kStreamBytesPerInEdge + sizeof(VItem))) +
                                   " bytes of stream slots beyond the resident arrays");
        uint32_t j = i;
        while (j < nitems && fits(std::max(end, items[j].in_end), j - i + 1)) {
            end = std::max(end, items[j].in_end);
            ++j;
        }
        c.count = j - i;
        c.span = end - c.base;
        for (uint32_t k = i; k < j; ++k) {
            items[k].in_begin -= c.base;
            items[k].in_end -= c.base;
        }
        P->max_items = std::max(P->max_items, c.count);
        P->slot_edges = std::max<uint64_t>(P->slot_edges, c.span);
        P->chunks.push_back(c);
        i = j;
    }
    if ((uint64_t)P->grid * P->chunks.size() * 8 > kPartialsReserve)
        fail(PGB_E_BUDGET, "device_budget leaves stream slots too small: " + std::to_string(P->chunks.size()) +
                               " chunks");
    // items in pinned memory so that their copies are asynchronous
    PGB_CUDA(cudaHostAlloc(&P->h_items, (size_t)nitems * sizeof(VItem), cudaHostAllocDefault));
    std::memcpy(P->h_items, items.data(), (size_t)nitems * sizeof(VItem));
    return P;
}

static std::shared_ptr<StreamPlan> get_plan(const pgb_blocks* b, uint32_t in_chunk, bool pv, uint32_t threads,
                                            uint64_t budget, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(b->plan_mu);
    auto P = std::static_pointer_cast<StreamPlan>(b->stream_plan);
    if (!P || P->in_chunk != in_chunk || P->budget != budget || P->pv != pv || P->threads_opt != threads) {
        P = make_plan(b, in_chunk, pv, threads, budget, s);
        b->stream_plan = P;
    }
    return P;
}

void run_streaming(const pgb_blocks* b, uint32_t in_chunk, bool pv, uint32_t threads, unsigned long long* tv,
                   uint64_t budget,
                   cudaStream_t s, DevBuf<unsigned long long>& partials, uint64_t& npartials, cudaEvent_t ev0,
                   cudaEvent_t ev1, uint64_t* streamed, uint32_t* nchunks_out, RunCtl* ctl, uint32_t core_e0) {
    npartials = 0;
    *streamed = 0;
    *nchunks_out = 0;
    const std::shared_ptr<StreamPlan> P = get_plan(b, in_chunk, pv, threads, budget, s);
    if (P->nitems == 0) {
        PGB_CUDA(cudaEventRecord(ev0, s));
        PGB_CUDA(cudaEventRecord(ev1, s));
        return;
    }
    const uint64_t slot_edges = P->slot_edges;
    const uint32_t max_items = P->max_items;
    const int grid = P->grid;
    DevBuf<unsigned long long> sxr[2] = {DevBuf<unsigned long long>(slot_edges, s),
                                         DevBuf<unsigned long long>(slot_edges, s)};
    DevBuf<uint32_t> stail[2] = {DevBuf<uint32_t>(slot_edges, s), DevBuf<uint32_t>(slot_edges, s)};
    DevBuf<VItem> sitems[2] = {DevBuf<VItem>(max_items, s), DevBuf<VItem>(max_items, s)};
    DevBuf<unsigned int> cursor(2, s);
    HashGraph hg[2];
    for (int k = 0; k < 2; ++k)
    {
        hg[k] = HashGraph{b->rowptr.ptr, b->col.ptr, nullptr, sxr[k].ptr, tv, b->n, stail[k].ptr};
        hg[k].colu = b->col.ptr;
        hg[k].core_e0 = core_e0;
    }
    npartials = (uint64_t)grid * P->chunks.size();
    partials.alloc(npartials, s);

    // copies on cs; chunk c counts on ks[c & 1] so that the launch of chunk
    // c + 1 fills the SMs that chunk c's last CTAs leave idle
    cudaStream_t cs = nullptr, s1 = nullptr;
    PGB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaEvent_t ready[2] = {}, freed[2] = {}, start = nullptr, done1 = nullptr;
    auto cleanup = [&] {
        if (cs) cudaStreamSynchronize(cs);
        if (s1) cudaStreamSynchronize(s1);
        for (int k = 0; k < 2; ++k) {
            if (ready[k]) cudaEventDestroy(ready[k]);
            if (freed[k]) cudaEventDestroy(freed[k]);
        }
        if (start) cudaEventDestroy(start);
        if (done1) cudaEventDestroy(done1);
        if (s1) cudaStreamDestroy(s1);
        cudaStreamDestroy(cs);
    };
    int rc = guard([&] {
        PGB_CUDA(cudaStreamCreateWithFlags(&s1, cudaStreamNonBlocking));
        for (int k = 0; k < 2; ++k) {
            PGB_CUDA(cudaEventCreateWithFlags(&ready[k], cudaEventDisableTiming));
            PGB_CUDA(cudaEventCreateWithFlags(&freed[k], cudaEventDisableTiming));
        }
        PGB_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
        PGB_CUDA(cudaEventCreateWithFlags(&done1, cudaEventDisableTiming));
        // the side streams start after everything already queued on s
        PGB_CUDA(cudaEventRecord(ev0, s));
        PGB_CUDA(cudaEventRecord(start, s));
        PGB_CUDA(cudaStreamWaitEvent(cs, start, 0));
        PGB_CUDA(cudaStreamWaitEvent(s1, start, 0));
        const cudaStream_t ks[2] = {s, s1};
        uint64_t bytes = 0;
        for (size_t c = 0; c < P->chunks.size(); ++c) {
            const int k = (int)(c & 1);
            const StreamPlan::Chunk& ch = P->chunks[c];
            if (c >= 2) PGB_CUDA(cudaStreamWaitEvent(cs, freed[k], 0));
            PGB_CUDA(cudaMemcpyAsync(sxr[k].ptr, b->h_xr + ch.base, (size_t)ch.span * 8, cudaMemcpyHostToDevice, cs));
            PGB_CUDA(cudaMemcpyAsync(stail[k].ptr, b->h_itail + ch.base, (size_t)ch.span * 4, cudaMemcpyHostToDevice,
                                     cs));
            PGB_CUDA(cudaMemcpyAsync(sitems[k].ptr, P->h_items + ch.first, (size_t)ch.count * sizeof(VItem),
                                     cudaMemcpyHostToDevice, cs));
            PGB_CUDA(cudaEventRecord(ready[k], cs));
            bytes += (uint64_t)ch.span * kStreamBytesPerInEdge + (uint64_t)ch.count * sizeof(VItem);
            PGB_CUDA(cudaStreamWaitEvent(ks[k], ready[k], 0));
            launch_hash(hg[k], sitems[k].ptr, ch.count, pv, ks[k], cursor.ptr + k, partials.ptr + c * grid, grid,
                        P->threads, ctl);
            PGB_CUDA(cudaEventRecord(freed[k], ks[k]));
        }
        PGB_CUDA(cudaEventRecord(done1, s1));
        PGB_CUDA(cudaStreamWaitEvent(s, done1, 0));
        PGB_CUDA(cudaEventRecord(ev1, s));
        *streamed = bytes;
        *nchunks_out = (uint32_t)P->chunks.size();
        // the slot buffers live on s; the pinned items must outlive the copies
        PGB_CUDA(cudaStreamSynchronize(s));
    });
    cleanup();
    if (rc != PGB_OK) fail(rc, pgb_last_error());
}

// ----------------------------------------------------------- column tier
//
// pgb_blocks_offload_columns moves the columns too, so that the device keeps
// only row offsets, the rank permutation and the counters (about 24 bytes per
// vertex).  The columns stay addressable by row block: row block i (ranks
// [c_i, c_{i+1})) is the contiguous column range [rowptr[c_i],
// rowptr[c_{i+1})), copied as one slice.  The in-edge index is re-sorted by
// (tail block, head, tail), so that the in-edges from tail block i into head
// block j (a block pair, the (A_ij, A_j*) part of the block-lists of Section
// 3.6) are contiguous.  A piece is at most kPieceInEdges in-edges of one
// block pair, with its work items built once at offload.  A run keeps a
// cache of column slices on the device (as many as the budget allows, least
// recently used evicted, never one that the current tasks need) and counts
// the pieces head-block group by head-block group: the group's head slices
// stay resident while the tail slices pass through.

constexpr uint64_t kPieceInEdges = 1ull << 21;

struct ColPiece {
    uint32_t i, j;      // tail block, head block
    uint64_t e0, e1;    // in-edges [e0, e1) of the tail-block-major index
    uint64_t it0, it1;  // work items [it0, it1)
};

struct ColPlan {
    uint32_t* h_col = nullptr;  // m + 16 columns (zero padded), pinned
    unsigned long long* h_bx = nullptr;  // index by (tail block, head, tail): tail-row range, pinned
    uint32_t* h_bt = nullptr;            // the tails, pinned
    VItem* h_items = nullptr;            // every piece's work items, pinned
    uint64_t nitems = 0;
    std::vector<ColPiece> pieces;
    uint32_t pc = 0;                            // row ranges (slices) of the columns
    std::vector<uint32_t> cuts;                 // pc + 1 rank cuts of those ranges
    std::vector<uint32_t> slice_lo, slice_len;  // per row range: first column (a multiple of 8), length
    ~ColPlan() {
        if (h_col) cudaFreeHost(h_col);
        if (h_bx) cudaFreeHost(h_bx);
        if (h_bt) cudaFreeHost(h_bt);
        if (h_items) cudaFreeHost(h_items);
    }
};

__device__ __forceinline__ uint32_t block_of(const uint32_t* __restrict__ cuts, uint32_t p, uint32_t r) {
    uint32_t lo = 0, hi = p;  // largest t with cuts[t] <= r
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (cuts[mid] <= r) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_tail_blocks(const uint32_t* __restrict__ itail, uint64_t m, const uint32_t* __restrict__ cuts,
                              uint32_t p, uint32_t* __restrict__ key, uint32_t* __restrict__ idx) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        key[i] = block_of(cuts, p, itail[i]);
        idx[i] = (uint32_t)i;
    }
}

// Gather the index in tail-block-major order: bx, bt, and the head of each
// in-edge (the column at the edge's CSR position).
__global__ void k_gather_block_major(const uint32_t* __restrict__ perm, uint64_t m,
                                     const unsigned long long* __restrict__ xr, const uint32_t* __restrict__ itail,
                                     const uint32_t* __restrict__ col, unsigned long long* __restrict__ bx,
                                     uint32_t* __restrict__ bt, uint32_t* __restrict__ bh) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += stride) {
        const uint32_t q = perm[k];
        const unsigned long long x = xr[q];
        bx[k] = x;
        bt[k] = itail[q];
        bh[k] = col[(uint32_t)x - 1];
    }
}

// bounds[i * (p + 1) + j] = first position of tail block i's section whose
// head is >= cuts[j] (the section [sec[i], sec[i+1]) is sorted by head);
// sec[i] = first position with key >= i.
__global__ void k_pair_bounds(const uint32_t* __restrict__ key, const uint32_t* __restrict__ bh, uint64_t m,
                              const uint32_t* __restrict__ cuts, uint32_t p, uint64_t* __restrict__ bounds) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p * (p + 1)) return;
    const uint32_t i = t / (p + 1), j = t % (p + 1);
    auto first_key = [&](uint32_t v) {
        uint64_t lo = 0, n = m;
        while (n > 0) {
            const uint64_t half = n >> 1;
            if (key[lo + half] < v) { lo += half + 1; n -= half + 1; } else { n = half; }
        }
        return lo;
    };
    const uint64_t s0 = first_key(i), s1 = first_key(i + 1);
    uint64_t lo = s0, n = s1 - s0;
    const uint32_t target = cuts[j];
    while (n > 0) {
        const uint64_t half = n >> 1;
        if (bh[lo + half] < target) { lo += half + 1; n -= half + 1; } else { n = half; }
    }
    bounds[t] = j == p ? s1 : lo;
}

// lc[v - w0] = in-edges of [e0, e1) whose head is < v, for v in [w0, w0 + len).
__global__ void k_local_colptr(const uint32_t* __restrict__ bh, uint64_t e0, uint64_t e1, uint32_t w0, uint32_t len,
                               uint32_t* __restrict__ lc) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= len) return;
    const uint32_t v = w0 + t;
    uint64_t lo = e0, n = e1 - e0;
    while (n > 0) {
        const uint64_t half = n >> 1;
        if (bh[lo + half] < v) { lo += half + 1; n -= half + 1; } else { n = half; }
    }
    lc[t] = (uint32_t)(lo - e0);
}

__global__ void k_gather_u32(const uint32_t* __restrict__ src, const uint64_t* __restrict__ at, uint32_t k,
                             uint32_t* __restrict__ out) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < k) out[t] = src[at[t]];
}

// Cuts of `pc` row ranges with about equal edges: cut[t] = least rank r with
// rowptr[r] * pc >= t * m (cut[pc] = n).
__global__ void k_col_cuts(const uint32_t* __restrict__ rowptr, uint32_t n, uint64_t m, uint32_t pc,
                           uint32_t* __restrict__ cuts, uint32_t* __restrict__ pos) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > pc) return;
    uint32_t lo = 0, hi = n;
    if (t == pc) {
        lo = n;
    } else {
        while (lo < hi) {
            const uint32_t mid = lo + (hi - lo) / 2;
            if ((uint64_t)rowptr[mid] * pc < (uint64_t)t * m) lo = mid + 1; else hi = mid;
        }
    }
    cuts[t] = lo;
    pos[t] = rowptr[lo];
}

static std::shared_ptr<ColPlan> build_col_plan(pgb_blocks* b, uint32_t pc, cudaStream_t s) {
    auto P = std::make_shared<ColPlan>();
    const uint64_t m = b->m;
    const uint32_t n = b->n;
    const uint32_t p = pc;
    P->pc = pc;
    // the row ranges of the slices and their column spans
    DevBuf<uint32_t> dcuts(p + 1, s);
    {
        DevBuf<uint32_t> dpos(p + 1, s);
        k_col_cuts<<<(p + 1 + 255) / 256, 256, 0, s>>>(b->rowptr.ptr, n, m, p, dcuts.ptr, dpos.ptr);
        PGB_CHECK_LAUNCH("k_col_cuts");
        std::vector<uint32_t> pos(p + 1);
        P->cuts.resize(p + 1);
        PGB_CUDA(cudaMemcpyAsync(pos.data(), dpos.ptr, (p + 1) * 4, cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaMemcpyAsync(P->cuts.data(), dcuts.ptr, (p + 1) * 4, cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaStreamSynchronize(s));
        P->slice_lo.resize(p);
        P->slice_len.resize(p);
        for (uint32_t i = 0; i < p; ++i) {
            const uint32_t lo = pos[i] & ~7u;
            const uint32_t hi = ((pos[i + 1] + 7) & ~7u) + 8;  // aligned 32-byte loads may read past the row
            P->slice_lo[i] = lo;
            P->slice_len[i] = hi - lo;
        }
    }
    PGB_CUDA(cudaHostAlloc(&P->h_col, (size_t)(m + 16) * 4, cudaHostAllocDefault));
    std::memset(P->h_col + m, 0, 16 * 4);
    if (m) PGB_CUDA(cudaMemcpyAsync(P->h_col, b->col.ptr, (size_t)m * 4, cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaHostAlloc(&P->h_bx, (size_t)std::max<uint64_t>(m, 1) * 8, cudaHostAllocDefault));
    PGB_CUDA(cudaHostAlloc(&P->h_bt, (size_t)std::max<uint64_t>(m, 1) * 4, cudaHostAllocDefault));
    if (m == 0) {
        PGB_CUDA(cudaStreamSynchronize(s));
        return P;
    }
    // tail-block-major order: a stable sort of the head-major index by the
    // tail's block keeps the head order (and each head's tail order) inside
    // each block
    DevBuf<uint32_t> itail(m, s);
    k_gather_tails<<<grid_for(m), 256, 0, s>>>(b->xr.ptr, m, b->rowidx.ptr, itail.ptr);
    PGB_CHECK_LAUNCH("k_gather_tails");
    DevBuf<uint32_t> key(m, s), key2(m, s), idx(m, s), idx2(m, s);
    k_tail_blocks<<<grid_for(m), 256, 0, s>>>(itail.ptr, m, dcuts.ptr, p, key.ptr, idx.ptr);
    PGB_CHECK_LAUNCH("k_tail_blocks");
    cub::DoubleBuffer<uint32_t> dk(key.ptr, key2.ptr), dv(idx.ptr, idx2.ptr);
    {
        Scratch scratch;
        size_t tmp = 0;
        const int bits = num_bits(p > 0 ? p - 1 : 0);
        PGB_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp, dk, dv, (int64_t)m, 0, bits, s));
        void* t = scratch.get(tmp, s);
        PGB_CUDA(cub::DeviceRadixSort::SortPairs(t, tmp, dk, dv, (int64_t)m, 0, bits, s));
    }
    const uint32_t* skey = dk.Current();
    DevBuf<unsigned long long> bx(m, s);
    DevBuf<uint32_t> bt(m, s), bh(m, s);
    k_gather_block_major<<<grid_for(m), 256, 0, s>>>(dv.Current(), m, b->xr.ptr, itail.ptr, b->col.ptr, bx.ptr,
                                                     bt.ptr, bh.ptr);
    PGB_CHECK_LAUNCH("k_gather_block_major");
    DevBuf<uint64_t> bounds((size_t)p * (p + 1), s);
    k_pair_bounds<<<(p * (p + 1) + 255) / 256, 256, 0, s>>>(skey, bh.ptr, m, dcuts.ptr, p, bounds.ptr);
    PGB_CHECK_LAUNCH("k_pair_bounds");
    std::vector<uint64_t> hb((size_t)p * (p + 1));
    PGB_CUDA(cudaMemcpyAsync(hb.data(), bounds.ptr, hb.size() * 8, cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaMemcpyAsync(P->h_bx, bx.ptr, (size_t)m * 8, cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaMemcpyAsync(P->h_bt, bt.ptr, (size_t)m * 4, cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaStreamSynchronize(s));
    key.release();
    key2.release();
    idx.release();
    idx2.release();
    itail.release();
    bx.release();
    bt.release();
    // pieces: at most kPieceInEdges in-edges of one block pair (i, j), with
    // their heads' first and last ranks read back in one copy
    std::vector<std::pair<uint64_t, uint64_t>> ranges;
    std::vector<std::pair<uint32_t, uint32_t>> pairs;
    for (uint32_t i = 0; i < p; ++i)
        for (uint32_t j = i; j < p; ++j) {
            const uint64_t a = hb[(size_t)i * (p + 1) + j], z = hb[(size_t)i * (p + 1) + j + 1];
            for (uint64_t e = a; e < z; e += kPieceInEdges) {
                ranges.push_back({e, std::min(z, e + kPieceInEdges)});
                pairs.push_back({i, j});
            }
        }
    const uint32_t np = (uint32_t)ranges.size();
    std::vector<uint64_t> ends(2 * (size_t)np);
    for (uint32_t k = 0; k < np; ++k) {
        ends[2 * k] = ranges[k].first;
        ends[2 * k + 1] = ranges[k].second - 1;
    }
    std::vector<uint32_t> heads(2 * (size_t)np);
    if (np) {
        DevBuf<uint64_t> dends(ends.size(), s);
        DevBuf<uint32_t> dheads(ends.size(), s);
        PGB_CUDA(cudaMemcpyAsync(dends.ptr, ends.data(), ends.size() * 8, cudaMemcpyHostToDevice, s));
        k_gather_u32<<<(unsigned)((ends.size() + 255) / 256), 256, 0, s>>>(bh.ptr, dends.ptr, (uint32_t)ends.size(),
                                                                          dheads.ptr);
        PGB_CHECK_LAUNCH("k_gather_u32");
        PGB_CUDA(cudaMemcpyAsync(heads.data(), dheads.ptr, heads.size() * 4, cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaStreamSynchronize(s));
    }
    std::vector<VItem> all;
    DevBuf<uint32_t> lc;
    for (uint32_t k = 0; k < np; ++k) {
        const uint64_t e0 = ranges[k].first, e1 = ranges[k].second;
        const uint32_t h0 = heads[2 * k], h1 = heads[2 * k + 1] + 1;
        const uint32_t w0 = h0 & ~31u;
        const uint32_t nwin = (h1 - w0 + 31) / 32;
        const uint32_t len = nwin * 32 + 1;
        if (lc.count < len) lc.alloc(len, s);
        k_local_colptr<<<(len + 255) / 256, 256, 0, s>>>(bh.ptr, e0, e1, w0, len, lc.ptr);
        PGB_CHECK_LAUNCH("k_local_colptr");
        // items that fit either CTA shape: the smaller table capacity
        const ItemSpace sp{b->rowptr.ptr, lc.ptr, b->col.ptr, w0, 0, w0, nwin, n, 1024, 131072};
        DevBuf<VItem> its;
        const uint32_t ni = build_hash_items_in(sp, 0, s, its);
        ColPiece pc{pairs[k].first, pairs[k].second, e0, e1, all.size(), all.size() + ni};
        const size_t old = all.size();
        all.resize(old + ni);
        if (ni) PGB_CUDA(cudaMemcpyAsync(all.data() + old, its.ptr, (size_t)ni * sizeof(VItem), cudaMemcpyDeviceToHost,
                                         s));
        PGB_CUDA(cudaStreamSynchronize(s));
        P->pieces.push_back(pc);
    }
    P->nitems = all.size();
    PGB_CUDA(cudaHostAlloc(&P->h_items, std::max<size_t>(all.size(), 1) * sizeof(VItem), cudaHostAllocDefault));
    if (!all.empty()) std::memcpy(P->h_items, all.data(), all.size() * sizeof(VItem));
    return P;
}

// Device bytes a column-streamed run holds besides its cache and piece slots.
static uint64_t col_resident_bytes(const pgb_blocks* b, bool pv) {
    const uint64_t n = b->n;
    return 4 * (n + 1) + 4 * n + 4 * ((uint64_t)b->p + 1) + (pv ? 16 * n : 0) + kPartialsReserve;
}

__global__ void k_add_partials(const unsigned long long* __restrict__ partials, uint32_t grid,
                               unsigned long long* __restrict__ acc) {
    __shared__ unsigned long long red[32];
    unsigned long long sum = 0;
    for (uint32_t i = threadIdx.x; i < grid; i += blockDim.x) sum += partials[i];
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x < 32) {
        sum = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
        if (threadIdx.x == 0) *acc += sum;
    }
}

// Sizes of a column-streamed run: the largest slice (entries), piece
// (in-edges, items), the launch grid, and the bytes held besides the slices.
struct ColSizes {
    uint64_t max_slice = 0, max_edges = 0, max_items = 0, fixed = 0;
    int grid = 0, threads = 128;
};

static ColSizes col_sizes(const pgb_blocks* b, bool pv, uint32_t threads) {
    const ColPlan& P = *std::static_pointer_cast<ColPlan>(b->col_plan);
    ColSizes z;
    for (uint32_t i = 0; i < P.pc; ++i) z.max_slice = std::max<uint64_t>(z.max_slice, P.slice_len[i]);
    for (const ColPiece& c : P.pieces) {
        z.max_edges = std::max(z.max_edges, c.e1 - c.e0);
        z.max_items = std::max(z.max_items, c.it1 - c.it0);
    }
    // pieces hold one tail block's in-edges, so items are small: the
    // 128-thread shape serves them better at every size measured
    z.threads = threads ? (int)threads : 128;
    z.grid = hash_grid(pv, z.threads);
    z.fixed = col_resident_bytes(b, pv) + 2 * (std::max<uint64_t>(z.max_edges, 1) * 12 +
                                               std::max<uint64_t>(z.max_items, 1) * sizeof(VItem)) +
              2ull * z.grid * 8 + 16;
    return z;
}

void run_column_streaming(const pgb_blocks* b, bool pv, uint32_t threads, unsigned long long* tv, uint64_t budget,
                          cudaStream_t s,
                          DevBuf<unsigned long long>& partials, uint64_t& npartials, cudaEvent_t ev0,
                          cudaEvent_t ev1, uint64_t* streamed, uint32_t* npieces_out, uint32_t* loads_out,
                          RunCtl* ctl) {
    const ColPlan& P = *std::static_pointer_cast<ColPlan>(b->col_plan);
    const uint32_t p = P.pc;
    npartials = 2;
    partials.alloc(2, s);
    PGB_CUDA(cudaMemsetAsync(partials.ptr, 0, 16, s));
    *streamed = 0;
    *npieces_out = (uint32_t)P.pieces.size();
    *loads_out = 0;
    if (P.pieces.empty()) {
        PGB_CUDA(cudaEventRecord(ev0, s));
        PGB_CUDA(cudaEventRecord(ev1, s));
        return;
    }
    const ColSizes z = col_sizes(b, pv, threads);
    const uint64_t max_slice = z.max_slice, max_edges = z.max_edges, max_items = z.max_items;
    const int grid = z.grid;
    uint32_t C = p;  // slices the cache holds
    if (budget) {
        if (budget <= z.fixed)
            fail(PGB_E_BUDGET, "device_budget of " + std::to_string(budget) + " bytes does not cover the " +
                                   std::to_string(z.fixed) + " bytes of resident arrays and piece slots");
        C = (uint32_t)std::min<uint64_t>(p, (budget - z.fixed) / (max_slice * 4));
        if (C < std::min<uint32_t>(2, p))
            fail(PGB_E_BUDGET, "device_budget leaves room for " + std::to_string(C) + " column slices of " +
                                   std::to_string(max_slice * 4) + " bytes; two are needed");
    }
    // task order: head blocks in groups of G; the group's head slices stay
    // while the tail blocks pass, so each tail slice is loaded once per group
    // with four slices or more, the next piece's copies are issued before
    // this piece's launch (queue lookahead), which needs one more slice
    const bool look = C >= 4;
    const uint32_t G = look ? C - 2 : std::max<uint32_t>(1, C > 1 ? C - 1 : 1);
    std::vector<std::vector<uint32_t>> by_pair((size_t)p * p);
    for (uint32_t k = 0; k < P.pieces.size(); ++k) by_pair[(size_t)P.pieces[k].i * p + P.pieces[k].j].push_back(k);
    std::vector<uint32_t> order;
    for (uint32_t g0 = 0; g0 < p; g0 += G) {
        const uint32_t g1 = std::min(p, g0 + G);
        for (uint32_t i = 0; i < g1; ++i)
            for (uint32_t j = std::max(g0, i); j < g1; ++j)
                for (uint32_t k : by_pair[(size_t)i * p + j]) order.push_back(k);
    }

    // device buffers: C slice slots, two piece slots, per-stream partials
    std::vector<DevBuf<uint32_t>> slot(C);
    for (uint32_t k = 0; k < C; ++k) slot[k].alloc(max_slice, s);
    DevBuf<unsigned long long> px[2] = {DevBuf<unsigned long long>(std::max<uint64_t>(max_edges, 1), s),
                                        DevBuf<unsigned long long>(std::max<uint64_t>(max_edges, 1), s)};
    DevBuf<uint32_t> pt[2] = {DevBuf<uint32_t>(std::max<uint64_t>(max_edges, 1), s),
                              DevBuf<uint32_t>(std::max<uint64_t>(max_edges, 1), s)};
    DevBuf<VItem> pit[2] = {DevBuf<VItem>(std::max<uint64_t>(max_items, 1), s),
                            DevBuf<VItem>(std::max<uint64_t>(max_items, 1), s)};
    DevBuf<unsigned long long> part(2 * (size_t)grid, s);
    DevBuf<unsigned int> cursor(2, s);

    std::vector<int> slot_blk(C, -1), blk_slot(p, -1);
    std::vector<uint64_t> slot_tick(C, 0);
    cudaStream_t cs = nullptr, s1 = nullptr;
    std::vector<cudaEvent_t> evs;  // every event made here, destroyed at the end
    auto mk = [&]() {
        cudaEvent_t e = nullptr;
        PGB_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        evs.push_back(e);
        return e;
    };
    std::vector<cudaEvent_t> slot_ready(C), slot_used0(C), slot_used1(C);
    std::vector<bool> used0(C, false), used1(C, false);
    cudaEvent_t piece_ready[2], piece_done[2], start, done1;
    auto cleanup = [&] {
        if (cs) cudaStreamSynchronize(cs);
        if (s1) cudaStreamSynchronize(s1);
        for (cudaEvent_t e : evs) cudaEventDestroy(e);
        if (s1) cudaStreamDestroy(s1);
        if (cs) cudaStreamDestroy(cs);
    };
    int rc = guard([&] {
        PGB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        PGB_CUDA(cudaStreamCreateWithFlags(&s1, cudaStreamNonBlocking));
        for (uint32_t k = 0; k < C; ++k) {
            slot_ready[k] = mk();
            slot_used0[k] = mk();
            slot_used1[k] = mk();
        }
        for (int k = 0; k < 2; ++k) {
            piece_ready[k] = mk();
            piece_done[k] = mk();
        }
        start = mk();
        done1 = mk();
        PGB_CUDA(cudaEventRecord(ev0, s));
        PGB_CUDA(cudaEventRecord(start, s));
        PGB_CUDA(cudaStreamWaitEvent(cs, start, 0));
        PGB_CUDA(cudaStreamWaitEvent(s1, start, 0));
        const cudaStream_t ks[2] = {s, s1};
        uint64_t tick = 0, bytes = 0;
        uint32_t loads = 0;
        // make block `blk` resident, never evicting the blocks in `keep`
        auto acquire = [&](uint32_t blk, const std::vector<uint32_t>& keep) -> uint32_t {
            if (blk_slot[blk] >= 0) {
                slot_tick[blk_slot[blk]] = ++tick;
                return (uint32_t)blk_slot[blk];
            }
            int victim = -1;
            for (uint32_t k = 0; k < C; ++k) {
                if (slot_blk[k] >= 0 && std::find(keep.begin(), keep.end(), (uint32_t)slot_blk[k]) != keep.end())
                    continue;
                if (victim < 0 || slot_blk[k] < 0 ||
                    (slot_blk[victim] >= 0 && slot_tick[k] < slot_tick[victim]))
                    victim = (int)k;
                if (slot_blk[victim] < 0) break;
            }
            if (victim < 0) fail(PGB_E_BUDGET, "column cache has no slot to evict");
            if (slot_blk[victim] >= 0) blk_slot[slot_blk[victim]] = -1;
            // the copy waits for every launch that read the evicted slice
            if (used0[victim]) PGB_CUDA(cudaStreamWaitEvent(cs, slot_used0[victim], 0));
            if (used1[victim]) PGB_CUDA(cudaStreamWaitEvent(cs, slot_used1[victim], 0));
            PGB_CUDA(cudaMemcpyAsync(slot[victim].ptr, P.h_col + P.slice_lo[blk], (size_t)P.slice_len[blk] * 4,
                                     cudaMemcpyHostToDevice, cs));
            PGB_CUDA(cudaEventRecord(slot_ready[victim], cs));
            bytes += (uint64_t)P.slice_len[blk] * 4;
            ++loads;
            slot_blk[victim] = (int)blk;
            blk_slot[blk] = victim;
            slot_tick[victim] = ++tick;
            return (uint32_t)victim;
        };
        std::vector<uint32_t> ssj(order.size()), ssi(order.size());
        // copies of piece t: its slices (never evicting those of the piece
        // staged before it, nor its head group's) and its index and items
        auto stage = [&](size_t t) {
            const ColPiece& c = P.pieces[order[t]];
            const int k = (int)(t & 1);
            const uint32_t G0 = (c.j / G) * G, G1 = std::min(p, G0 + G);
            std::vector<uint32_t> keep;
            for (uint32_t jj = G0; jj < G1; ++jj)
                if (blk_slot[jj] >= 0) keep.push_back(jj);
            keep.push_back(c.i);
            keep.push_back(c.j);
            if (look && t > 0) {  // staged ahead of the launch of piece t - 1
                keep.push_back(P.pieces[order[t - 1]].i);
                keep.push_back(P.pieces[order[t - 1]].j);
            }
            ssj[t] = acquire(c.j, keep);
            ssi[t] = acquire(c.i, keep);
            if (t >= 2) PGB_CUDA(cudaStreamWaitEvent(cs, piece_done[k], 0));
            const uint64_t ne = c.e1 - c.e0, ni = c.it1 - c.it0;
            PGB_CUDA(cudaMemcpyAsync(px[k].ptr, P.h_bx + c.e0, ne * 8, cudaMemcpyHostToDevice, cs));
            PGB_CUDA(cudaMemcpyAsync(pt[k].ptr, P.h_bt + c.e0, ne * 4, cudaMemcpyHostToDevice, cs));
            if (ni)
                PGB_CUDA(cudaMemcpyAsync(pit[k].ptr, P.h_items + c.it0, ni * sizeof(VItem), cudaMemcpyHostToDevice,
                                         cs));
            PGB_CUDA(cudaEventRecord(piece_ready[k], cs));
            bytes += ne * 12 + ni * sizeof(VItem);
        };
        // the counting launch of piece t on stream t & 1
        auto launch = [&](size_t t) {
            const ColPiece& c = P.pieces[order[t]];
            const int k = (int)(t & 1);
            const cudaStream_t ss = ks[k];
            const uint32_t sj = ssj[t], si = ssi[t];
            const uint64_t ni = c.it1 - c.it0;
            PGB_CUDA(cudaStreamWaitEvent(ss, piece_ready[k], 0));
            PGB_CUDA(cudaStreamWaitEvent(ss, slot_ready[sj], 0));
            PGB_CUDA(cudaStreamWaitEvent(ss, slot_ready[si], 0));
            HashGraph Gr{b->rowptr.ptr, slot[sj].ptr, nullptr, px[k].ptr, tv, b->n, pt[k].ptr};
            Gr.vbase = P.slice_lo[c.j];
            Gr.colu = slot[si].ptr;
            Gr.ubase = P.slice_lo[c.i];
            if (ni) {
                launch_hash(Gr, pit[k].ptr, (uint32_t)ni, pv, ss, cursor.ptr + k, part.ptr + (size_t)k * grid, grid,
                            z.threads, ctl);
                k_add_partials<<<1, 256, 0, ss>>>(part.ptr + (size_t)k * grid, (uint32_t)grid, partials.ptr + k);
                PGB_CHECK_LAUNCH("k_add_partials");
            }
            PGB_CUDA(cudaEventRecord(piece_done[k], ss));
            for (uint32_t q : {sj, si}) {
                PGB_CUDA(cudaEventRecord(k ? slot_used1[q] : slot_used0[q], ss));
                (k ? used1 : used0)[q] = true;
            }
        };
        if (look) {
            if (!order.empty()) stage(0);
            for (size_t t = 0; t < order.size(); ++t) {
                if (t + 1 < order.size()) stage(t + 1);
                launch(t);
            }
        } else {
            for (size_t t = 0; t < order.size(); ++t) {
                stage(t);
                launch(t);
            }
        }
        PGB_CUDA(cudaEventRecord(done1, s1));
        PGB_CUDA(cudaStreamWaitEvent(s, done1, 0));
        PGB_CUDA(cudaEventRecord(ev1, s));
        *streamed = bytes;
        *loads_out = loads;
        // the slots live on s; the pinned sources must outlive the copies
        PGB_CUDA(cudaStreamSynchronize(s));
    });
    cleanup();
    if (rc != PGB_OK) fail(rc, pgb_last_error());
}

const uint32_t* offloaded_columns(const pgb_blocks* b) {
    return b->cols_offloaded ? std::static_pointer_cast<ColPlan>(b->col_plan)->h_col : nullptr;
}

}  // namespace pgb

using namespace pgb;

extern "C" {

int pgb_blocks_resident_bytes(const pgb_blocks* b, int per_vertex, uint64_t* bytes) {
    return guard([&] {
        if (!b || !bytes) fail(PGB_E_INVAL, "NULL argument");
        *bytes = b->cols_offloaded ? col_resident_bytes(b, per_vertex != 0) : resident_bytes(b, per_vertex != 0);
    });
}

int pgb_blocks_cache_budget(const pgb_blocks* b, int per_vertex, uint32_t slices, uint64_t* budget) {
    return guard([&] {
        if (!b || !budget) fail(PGB_E_INVAL, "NULL argument");
        if (!b->cols_offloaded) fail(PGB_E_STATE, "the columns are not offloaded");
        const ColSizes z = col_sizes(b, per_vertex != 0, 0);
        const uint32_t pc = std::static_pointer_cast<ColPlan>(b->col_plan)->pc;
        *budget = z.fixed + (uint64_t)std::min(slices, pc) * z.max_slice * 4;
    });
}

int pgb_blocks_offload_columns(pgb_blocks* b, uint32_t slices, void* stream) {
    return guard([&] {
        if (!b) fail(PGB_E_INVAL, "blocks is NULL");
        if (slices > 1024) fail(PGB_E_INVAL, "slices must be at most 1024");
        if (b->cols_offloaded) return;
        if (b->offloaded) fail(PGB_E_STATE, "the in-edge index is already offloaded; offload the columns first");
        cudaStream_t s = (cudaStream_t)stream;
        const uint32_t pc = std::max<uint32_t>(1, std::min<uint32_t>(slices ? slices : b->p, std::max(b->n, 1u)));
        std::shared_ptr<ColPlan> P = build_col_plan(b, pc, s);
        {
            std::lock_guard<std::mutex> lk(b->plan_mu);
            b->run_plans.clear();
            b->stream_plan.reset();
        }
        b->xr.release();
        b->rowidx.release();
        b->col.release();
        b->colptr.release();
        {
            std::lock_guard<std::mutex> lk(b->bedge_mu);
            b->bedge.release();
            b->bedge_ready = false;
        }
        PGB_CUDA(cudaStreamSynchronize(s));
        b->col_plan = P;
        b->offloaded = true;
        b->cols_offloaded = true;
    });
}

int pgb_blocks_offload(pgb_blocks* b, void* stream) {
    return guard([&] {
        if (!b) fail(PGB_E_INVAL, "blocks is NULL");
        if (b->offloaded) return;
        cudaStream_t s = (cudaStream_t)stream;
        const uint64_t m = b->m;
        PGB_CUDA(cudaHostAlloc(&b->h_xr, std::max<uint64_t>(m, 1) * 8, cudaHostAllocDefault));
        PGB_CUDA(cudaHostAlloc(&b->h_itail, std::max<uint64_t>(m, 1) * 4, cudaHostAllocDefault));
        if (m) {
            DevBuf<uint32_t> itail(m, s);
            k_gather_tails<<<grid_for(m), 256, 0, s>>>(b->xr.ptr, m, b->rowidx.ptr, itail.ptr);
            PGB_CHECK_LAUNCH("k_gather_tails");
            PGB_CUDA(cudaMemcpyAsync(b->h_xr, b->xr.ptr, m * 8, cudaMemcpyDeviceToHost, s));
            PGB_CUDA(cudaMemcpyAsync(b->h_itail, itail.ptr, m * 4, cudaMemcpyDeviceToHost, s));
            PGB_CUDA(cudaStreamSynchronize(s));
        }
        // the in-edge index leaves the device, and so do the arrays only the
        // edge-wise kernels use
        {
            // captured runs point at the arrays released below
            std::lock_guard<std::mutex> lk(b->plan_mu);
            b->run_plans.clear();
        }
        b->xr.release();
        b->rowidx.release();
        {
            std::lock_guard<std::mutex> lk(b->bedge_mu);
            b->bedge.release();
            b->bedge_ready = false;
        }
        PGB_CUDA(cudaStreamSynchronize(s));
        b->offloaded = true;
    });
}

}  // extern "C"
