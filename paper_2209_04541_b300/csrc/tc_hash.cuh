// Middle-vertex hash variant: entry used by the run orchestration.
#pragma once

#include "internal.cuh"

namespace pgb {

struct HashGraph {
    const uint32_t* __restrict__ rowptr;
    const uint32_t* __restrict__ col;
    const uint32_t* __restrict__ rowidx;
    const uint32_t* __restrict__ colptr;
    const unsigned long long* __restrict__ xr;
    unsigned long long* __restrict__ tv;  // per-vertex counts, rank space (may be null)
    uint32_t n;                           // vertices
    const uint32_t* __restrict__ itail = nullptr;  // tail of each in-edge (streamed runs), else null
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
    uint32_t pad;         // keeps items 32 bytes
};

// Work items of one partitioned graph; returns their number (synchronises
// `s` once to learn it).  in_chunk: in-edges per item (0 = default).
uint32_t build_hash_items(const pgb_blocks* b, uint32_t in_chunk, cudaStream_t s, DevBuf<VItem>& items);

// CTAs of a persistent launch on the current device.
int hash_grid(bool pv);

// One persistent launch over `nitems` work items of graph G; partials must
// hold `grid` entries and receive one total per CTA.
void launch_hash(const HashGraph& G, const VItem* items, uint32_t nitems, bool pv, cudaStream_t s,
                 unsigned int* cursor, unsigned long long* partials, int grid);

// Streamed run over blocks whose in-edge index is in pinned host memory:
// chunks of work items whose in-edges fit two device slots within `budget`
// bytes (0 = 1 GiB slots), copied on a side stream while the previous chunk
// counts on `s`.  Returns after the work completes.
void run_streaming(const pgb_blocks* b, uint32_t in_chunk, bool pv, unsigned long long* tv, uint64_t budget,
                   cudaStream_t s, DevBuf<unsigned long long>& partials, uint64_t& npartials, cudaEvent_t ev0,
                   cudaEvent_t ev1, uint64_t* streamed, uint32_t* nchunks);

}  // namespace pgb
