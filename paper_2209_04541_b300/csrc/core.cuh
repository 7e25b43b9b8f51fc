// Dense count of the top block of the degree order (core.cu).
#pragma once

#include <cuda_fp16.h>

#include "internal.cuh"

namespace pgb {

// The top K ranks [c0, n) as one dense block: its 0/1 adjacency A (K x K,
// fp16, symmetric), a column strip of A·A (fp32), per-vertex sums.
struct CorePlan {
    uint32_t K = 0, c0 = 0, e0 = 0, tile = 0;  // e0 = rowptr[c0]: the block's first CSR position
    uint64_t m = 0;
    const uint32_t* rowptr = nullptr;  // the oriented graph's rows (rank space)
    const uint32_t* col = nullptr;
    DevBuf<__half> A;
    DevBuf<float> C;
    DevBuf<unsigned long long> S;
    DevBuf<unsigned char> workspace;  // cuBLAS workspace (graph capture needs one of the caller's)
};

// Lookups per tail-rank band of the top ranks: band i counts the lookups of
// in-edges whose tail has rank in [n - (i + 1) * kCoreBand, n - i * kCoreBand).
constexpr uint32_t kCoreBand = 1024;
constexpr uint32_t kCoreBands = 32;  // up to the top 32,768 ranks

// The block size the autotuner picks (0: no dense block) from the lookups
// per band (b->core_probes) and the GEMM's cost; opt > 0 asks for that many
// ranks (rounded up to a multiple of 256, at most n), opt < 0 for none.
uint32_t choose_core(const pgb_blocks* b, int32_t opt);

// Floating-point operations of the A·A strips for the top K ranks.
double core_flop(uint32_t K);

// Allocate and fill the plan for the top K ranks (synchronises s once).
void core_prepare(const pgb_blocks* b, uint32_t K, cudaStream_t s, CorePlan& P);

// Count the block's triangles: adds t[x] of its vertices into tv (rank
// space, may be null) and writes the block's total to *slot.  Capturable.
void core_enqueue(const CorePlan& P, unsigned long long* tv, unsigned long long* slot, cudaStream_t s);

// *to += *from on the device (one thread).
void core_add_total(const unsigned long long* from, unsigned long long* to, cudaStream_t s);

// Device bytes a plan for the top K ranks holds.
uint64_t core_bytes(uint32_t K);

// The per-band lookups of the top ranks (kCoreBands values), on the device.
void core_band_probes(const pgb_blocks* b, unsigned long long* bands, cudaStream_t s);

}  // namespace pgb
