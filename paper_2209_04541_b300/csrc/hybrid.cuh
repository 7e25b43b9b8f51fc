// Hybrid scheduler: the host kernel K_H and the cut-off (hybrid.cu).
#pragma once

#include "internal.cuh"

namespace pgb {

// Host parts under the cut-off: the lightest head parts (estimate: lookups
// plus in-edges) whose summed estimate stays within share_ppm / 10^6 of the
// total.  Entry j is 1 for a host part.
std::vector<uint8_t> host_parts_by_cutoff(const pgb_blocks* b, uint32_t share_ppm);

struct HostCountResult {
    uint64_t total = 0;     // triangles whose middle vertex lies in a host part
    uint64_t in_edges = 0;  // in-edges of the host parts
    uint32_t parts = 0;
    uint32_t threads = 0;
    float ms = 0;           // wall time of the host count (mirror copy included on first use)
    bool cancelled = false; // the cancel token was seen; counts are incomplete
};

// Count the host parts on `threads` host threads (0: all hardware threads).
// With per_vertex, the per-vertex counts (rank space) are appended to `adds`
// as (vertex, count) pairs (a vertex may appear more than once): the host
// parts are the light ones, so their contributions are sparse.  Copies the
// oriented graph to a host mirror on first use (synchronising s).
// In-edges whose tail row starts at CSR position core_e0 or later are left to
// the dense top block.
HostCountResult host_count_parts(const pgb_blocks* b, const std::vector<uint8_t>& host, uint32_t threads,
                                 bool per_vertex, std::vector<std::pair<uint32_t, uint32_t>>& adds,
                                 const pgb_cancel* cancel, cudaStream_t s, uint32_t core_e0 = 0xFFFFFFFFu);

}  // namespace pgb
