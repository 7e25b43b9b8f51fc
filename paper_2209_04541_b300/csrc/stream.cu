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
    return 4 * (n + 1) + 4 * (b->m + 4) + 4 * (n + 1) + 4 * n + 4 * ((uint64_t)b->p + 1) + (pv ? 16 * n : 0) +
           kPartialsReserve;
}

void run_streaming(const pgb_blocks* b, uint32_t in_chunk, bool pv, unsigned long long* tv, uint64_t budget,
                   cudaStream_t s, DevBuf<unsigned long long>& partials, uint64_t& npartials, cudaEvent_t ev0,
                   cudaEvent_t ev1, uint64_t* streamed, uint32_t* nchunks_out) {
    npartials = 0;
    *streamed = 0;
    *nchunks_out = 0;
    DevBuf<VItem> ditems;
    const uint32_t nitems = build_hash_items(b, 0, in_chunk, s, ditems);
    if (nitems == 0) {
        PGB_CUDA(cudaEventRecord(ev0, s));
        PGB_CUDA(cudaEventRecord(ev1, s));
        return;
    }
    // work items in in-edge order; a chunk is a run of items whose in-edge
    // span fits one slot
    std::vector<VItem> items(nitems);
    PGB_CUDA(cudaMemcpyAsync(items.data(), ditems.ptr, (size_t)nitems * sizeof(VItem), cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaStreamSynchronize(s));
    ditems.release();
    std::stable_sort(items.begin(), items.end(),
                     [](const VItem& x, const VItem& y) { return x.in_begin < y.in_begin; });
    // the budget covers everything the run holds on the device: the resident
    // arrays, the per-vertex counters, the per-launch partials (bounded by
    // kPartialsReserve) and the two stream slots
    const int grid = hash_grid(pv);
    const uint64_t resident = resident_bytes(b, pv);
    uint64_t slot_bytes = kDefaultSlotBytes;
    if (budget) {
        if (budget <= resident)
            fail(PGB_E_BUDGET, "device_budget of " + std::to_string(budget) + " bytes is below the " +
                                   std::to_string(resident) + " bytes the resident arrays need");
        slot_bytes = (budget - resident) / 2;
    }
    const uint64_t cap = slot_bytes / (kStreamBytesPerInEdge + sizeof(VItem));  // in-edges per slot
    struct Chunk {
        uint32_t first, count, base, span;
    };
    std::vector<Chunk> chunks;
    uint32_t max_items = 0;
    for (uint32_t i = 0; i < nitems;) {
        Chunk c{i, 0, items[i].in_begin, 0};
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
        max_items = std::max(max_items, c.count);
        chunks.push_back(c);
        i = j;
    }
    // items in pinned memory so their copies are asynchronous
    VItem* h_items = nullptr;
    PGB_CUDA(cudaHostAlloc(&h_items, (size_t)nitems * sizeof(VItem), cudaHostAllocDefault));
    std::unique_ptr<VItem, cudaError_t (*)(void*)> h_items_guard(h_items, cudaFreeHost);
    std::memcpy(h_items, items.data(), (size_t)nitems * sizeof(VItem));

    if ((uint64_t)grid * chunks.size() * 8 > kPartialsReserve)
        fail(PGB_E_BUDGET, "device_budget leaves stream slots too small: " + std::to_string(chunks.size()) +
                               " chunks");
    uint64_t slot_edges = 0;
    for (const Chunk& ch : chunks) slot_edges = std::max<uint64_t>(slot_edges, ch.span);
    DevBuf<unsigned long long> sxr[2] = {DevBuf<unsigned long long>(slot_edges, s),
                                         DevBuf<unsigned long long>(slot_edges, s)};
    DevBuf<uint32_t> stail[2] = {DevBuf<uint32_t>(slot_edges, s), DevBuf<uint32_t>(slot_edges, s)};
    DevBuf<VItem> sitems[2] = {DevBuf<VItem>(max_items, s), DevBuf<VItem>(max_items, s)};
    DevBuf<HashGraph> sg[2] = {DevBuf<HashGraph>(1, s), DevBuf<HashGraph>(1, s)};
    DevBuf<unsigned int> cursor[2] = {DevBuf<unsigned int>(1, s), DevBuf<unsigned int>(1, s)};
    HashGraph hg[2];
    for (int k = 0; k < 2; ++k) {
        hg[k] = HashGraph{b->rowptr.ptr, b->col.ptr, nullptr, b->colptr.ptr, sxr[k].ptr, tv, b->n, stail[k].ptr};
        PGB_CUDA(cudaMemcpyAsync(sg[k].ptr, &hg[k], sizeof(HashGraph), cudaMemcpyHostToDevice, s));
    }
    npartials = (uint64_t)grid * chunks.size();
    partials.alloc(npartials, s);

    cudaStream_t cs = nullptr;
    PGB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaEvent_t ready[2], freed[2], start;
    PGB_CUDA(cudaEventCreateWithFlags(&ready[0], cudaEventDisableTiming));
    PGB_CUDA(cudaEventCreateWithFlags(&ready[1], cudaEventDisableTiming));
    PGB_CUDA(cudaEventCreateWithFlags(&freed[0], cudaEventDisableTiming));
    PGB_CUDA(cudaEventCreateWithFlags(&freed[1], cudaEventDisableTiming));
    PGB_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    auto cleanup = [&] {
        cudaStreamSynchronize(cs);
        for (int k = 0; k < 2; ++k) {
            cudaEventDestroy(ready[k]);
            cudaEventDestroy(freed[k]);
        }
        cudaEventDestroy(start);
        cudaStreamDestroy(cs);
    };
    int rc = guard([&] {
        // the side stream starts after everything already queued on s
        PGB_CUDA(cudaEventRecord(start, s));
        PGB_CUDA(cudaStreamWaitEvent(cs, start, 0));
        PGB_CUDA(cudaEventRecord(ev0, s));
        uint64_t bytes = 0;
        for (size_t c = 0; c < chunks.size(); ++c) {
            const int k = (int)(c & 1);
            const Chunk& ch = chunks[c];
            if (c >= 2) PGB_CUDA(cudaStreamWaitEvent(cs, freed[k], 0));
            PGB_CUDA(cudaMemcpyAsync(sxr[k].ptr, b->h_xr + ch.base, (size_t)ch.span * 8, cudaMemcpyHostToDevice, cs));
            PGB_CUDA(cudaMemcpyAsync(stail[k].ptr, b->h_itail + ch.base, (size_t)ch.span * 4, cudaMemcpyHostToDevice,
                                     cs));
            PGB_CUDA(cudaMemcpyAsync(sitems[k].ptr, h_items + ch.first, (size_t)ch.count * sizeof(VItem),
                                     cudaMemcpyHostToDevice, cs));
            PGB_CUDA(cudaEventRecord(ready[k], cs));
            bytes += (uint64_t)ch.span * kStreamBytesPerInEdge + (uint64_t)ch.count * sizeof(VItem);
            PGB_CUDA(cudaStreamWaitEvent(s, ready[k], 0));
            launch_hash(sg[k].ptr, 1, sitems[k].ptr, ch.count, pv, s, cursor[k].ptr, partials.ptr + c * grid, grid);
            PGB_CUDA(cudaEventRecord(freed[k], s));
        }
        PGB_CUDA(cudaEventRecord(ev1, s));
        *streamed = bytes;
        *nchunks_out = (uint32_t)chunks.size();
        // the slot buffers and pinned items must outlive the queued work
        PGB_CUDA(cudaStreamSynchronize(s));
    });
    cleanup();
    if (rc != PGB_OK) fail(rc, pgb_last_error());
}

}  // namespace pgb

using namespace pgb;

extern "C" {

int pgb_blocks_resident_bytes(const pgb_blocks* b, int per_vertex, uint64_t* bytes) {
    return guard([&] {
        if (!b || !bytes) fail(PGB_E_INVAL, "NULL argument");
        *bytes = resident_bytes(b, per_vertex != 0);
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
