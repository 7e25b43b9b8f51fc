// Middle-vertex hash variant: entry used by the run orchestration.
#pragma once

#include "internal.cuh"

namespace pgb {

struct HashGraph {
    const uint32_t* __restrict__ rowptr;
    const uint32_t* __restrict__ col;     // rows of the middle vertices: entry q at col[q - vbase]
    const uint32_t* __restrict__ rowidx;
    const unsigned long long* __restrict__ xr;
    unsigned long long* __restrict__ tv;  // per-vertex counts, rank space (may be null)
    uint32_t n;                           // vertices
    const uint32_t* __restrict__ itail = nullptr;  // tail of each in-edge (streamed runs), else null
    const uint32_t* __restrict__ colu = nullptr;   // rows of the tails: entry q at colu[q - ubase]
    uint32_t vbase = 0, ubase = 0;                 // ubase is a multiple of 8 (32-byte loads)
    // in-edges whose tail-row position e (xr low word - 1) is at least this
    // are skipped: their triangles lie in the dense top block (core.cu)
    uint32_t core_e0 = 0xFFFFFFFFu;
};

// Where the item builder finds the heads of a set of in-edges: window w
// covers heads w0 + 32w .. w0 + 32w + 31; in-degrees come from
// colptr[v - cbase], out-rows from rowptr (global) and col[q - vbase].
struct ItemSpace {
    const uint32_t* rowptr;
    const uint32_t* colptr;
    const uint32_t* col;
    uint32_t cbase, vbase, w0, nwin, n;
    uint32_t keycap;       // table keys per item: 1024 (fits both CTA shapes) or 2048 (256 threads only)
    uint32_t bitmap_bits;  // a singleton range narrower than this is a bitmap (such vertices are never grouped)
    // optional filter: only heads v whose part j (cuts[j] <= v < cuts[j+1])
    // has part_hash[j] != 0 get work items (null: every head)
    const uint8_t* part_hash = nullptr;
    const uint32_t* cuts = nullptr;
    uint32_t p = 0;
};

// One work item of the middle-vertex kernel (built on the device).
struct VItem {
    uint32_t v0;          // first middle vertex (rank)
    uint32_t nv;          // consecutive middle vertices in the item (<= 32)
    uint32_t in_begin;    // in-edge range [in_begin, in_end) of the in-edge index
    uint32_t in_end;
    uint32_t lo, hi;      // third-vertex rank range
    uint16_t slots_log2;  // hash table size
    uint16_t clip;        // 1 when lists are clipped to [lo, hi)
    uint32_t mask;        // members with in-edges and out-edges in this item's index (bit t: v0 + t)
};

// Work items of one partitioned graph for the hash kernel with `threads`
// per CTA; returns their number (synchronises `s` once to learn it).
// in_chunk: in-edges per item (0 = the default for streamed runs, 4,096).
// part_hash (device, p bytes, may be null): only heads in parts with a
// non-zero entry get items; the other parts' triangles are left to the
// edge-wise kernel (per-part autotuning).
uint32_t build_hash_items(const pgb_blocks* b, uint32_t in_chunk, int threads, cudaStream_t s,
                          DevBuf<VItem>& items, const uint8_t* part_hash = nullptr);

// In-edges per work item of a resident run when the caller sets none: larger
// items amortise the per-item table build and barrier (measured 0.5% faster
// than 4,096 at R-MAT scales 22 and 24); streamed runs keep 4,096 so that
// their copy slots stay small.
constexpr uint32_t kResidentInChunk = 16384;

// The same over an item space (a range of heads with their own in-edge
// offsets); item in-edge ranges are positions in those offsets.
uint32_t build_hash_items_in(const ItemSpace& sp, uint32_t in_chunk, cudaStream_t s, DevBuf<VItem>& items);

// The graph view of a resident partition for the hash kernel.
HashGraph resident_hash_graph(const pgb_blocks* b, unsigned long long* tv);

// Threads per CTA of the hash kernel for a graph of n vertices (128 or 256;
// part of the run-level autotuner).
int hash_threads(uint32_t n);

// CTAs of a persistent launch of that shape on the current device.
int hash_grid(bool pv, int threads);

// One persistent launch over `nitems` work items of graph G; partials must
// hold `grid` entries and receive one total per CTA.  ctl (device memory,
// may be null): the run's stop word, read every kStopCheckEvery fetches.
void launch_hash(const HashGraph& G, const VItem* items, uint32_t nitems, bool pv, cudaStream_t s,
                 unsigned int* cursor, unsigned long long* partials, int grid, int threads, RunCtl* ctl);

// Streamed run over blocks whose in-edge index is in pinned host memory:
// chunks of work items whose in-edges fit two device slots within `budget`
// bytes (0 = 1 GiB slots), copied on a side stream while the previous chunk
// counts on `s`.  threads: CTA shape (0 = autotuned).  Returns after the
// work completes.
void run_streaming(const pgb_blocks* b, uint32_t in_chunk, bool pv, uint32_t threads, unsigned long long* tv,
                   uint64_t budget,
                   cudaStream_t s, DevBuf<unsigned long long>& partials, uint64_t& npartials, cudaEvent_t ev0,
                   cudaEvent_t ev1, uint64_t* streamed, uint32_t* nchunks, RunCtl* ctl,
                   uint32_t core_e0 = 0xFFFFFFFFu);  // in-edges at or after it left to the dense top block

// Run over blocks whose columns are offloaded too: pieces of block pairs
// (tail block, head block) with their column slices in a device cache that
// the budget sizes.  Returns after the work completes; partials gets two
// running totals.
void run_column_streaming(const pgb_blocks* b, bool pv, uint32_t threads, unsigned long long* tv, uint64_t budget,
                          cudaStream_t s,
                          DevBuf<unsigned long long>& partials, uint64_t& npartials, cudaEvent_t ev0,
                          cudaEvent_t ev1, uint64_t* streamed, uint32_t* npieces, uint32_t* slice_loads,
                          RunCtl* ctl);

}  // namespace pgb
