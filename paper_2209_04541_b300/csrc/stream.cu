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

// The chunking of one (work-item size, budget, per-vertex) setting, kept on
// the blocks handle: building it needs the items on the host once.
struct StreamPlan {
    struct Chunk {
        uint32_t first, count, base, span;  // items [first, first+count), in-edges [base, base+span)
    };
    uint32_t in_chunk = 0;
    uint64_t budget = 0;
    bool pv = false;
    int grid = 0;
    std::vector<Chunk> chunks;
    VItem* h_items = nullptr;  // pinned, in-edge ranges relative to their chunk's base
    uint32_t nitems = 0, max_items = 0;
    uint64_t slot_edges = 0;
    ~StreamPlan() {
        if (h_items) cudaFreeHost(h_items);
    }
};

static std::shared_ptr<StreamPlan> make_plan(const pgb_blocks* b, uint32_t in_chunk, bool pv, uint64_t budget,
                                             cudaStream_t s) {
    auto P = std::make_shared<StreamPlan>();
    P->in_chunk = in_chunk;
    P->budget = budget;
    P->pv = pv;
    P->grid = hash_grid(pv);
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
    const uint32_t nitems = build_hash_items(b, in_chunk, s, ditems);
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

static std::shared_ptr<StreamPlan> get_plan(const pgb_blocks* b, uint32_t in_chunk, bool pv, uint64_t budget,
                                            cudaStream_t s) {
    std::lock_guard<std::mutex> lk(b->plan_mu);
    auto P = std::static_pointer_cast<StreamPlan>(b->stream_plan);
    if (!P || P->in_chunk != in_chunk || P->budget != budget || P->pv != pv) {
        P = make_plan(b, in_chunk, pv, budget, s);
        b->stream_plan = P;
    }
    return P;
}

void run_streaming(const pgb_blocks* b, uint32_t in_chunk, bool pv, unsigned long long* tv, uint64_t budget,
                   cudaStream_t s, DevBuf<unsigned long long>& partials, uint64_t& npartials, cudaEvent_t ev0,
                   cudaEvent_t ev1, uint64_t* streamed, uint32_t* nchunks_out) {
    npartials = 0;
    *streamed = 0;
    *nchunks_out = 0;
    const std::shared_ptr<StreamPlan> P = get_plan(b, in_chunk, pv, budget, s);
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
        hg[k] = HashGraph{b->rowptr.ptr, b->col.ptr, nullptr, b->colptr.ptr, sxr[k].ptr, tv, b->n, stail[k].ptr};
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
            launch_hash(hg[k], sitems[k].ptr, ch.count, pv, ks[k], cursor.ptr + k, partials.ptr + c * grid, grid);
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
