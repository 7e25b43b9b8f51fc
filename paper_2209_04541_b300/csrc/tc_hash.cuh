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
};

struct HashRunStats {
    uint32_t items = 0;
    int grid = 0;
};

// Builds the work items and launches the persistent hash kernel on `s`
// between events ev0 and ev1; per-CTA totals land in `partials`.
// in_chunk: in-edges per work item (0 = default).
void run_hash(const pgb_blocks* b, const HashGraph& G, bool pv, uint32_t in_chunk, cudaStream_t s,
              DevBuf<unsigned long long>& partials, uint64_t& npartials, cudaEvent_t ev0, cudaEvent_t ev1,
              HashRunStats* stats);

}  // namespace pgb
