// Host kernel K_H of the hybrid scheduler (PGAbB Section 4.4).
//
// The paper's scheduler orders the tasks by their estimated work and hands
// the heavy ones to the GPU and the light ones to CPU threads; a cut-off
// keeps the CPUs off the heavy end.  Here a task is a head part V_j (the
// column block: every triangle whose middle vertex lies in V_j), its
// estimate is its lookups plus its in-edges, and the cut-off is a share of
// the total estimate: the host takes the lightest parts while their summed
// estimate stays within the share, the GPU counts the others in the same
// run.  Within the host parts, host threads take runs of heads from a shared
// counter (lightest part first).
//
// The host kernel counts the triangles of a head v the way the device's
// middle-vertex kernel does: for each in-edge (u, v), the entries of u's row
// after v that also lie in v's row close a triangle u < v < w.  Both lists
// are sorted ranks; the shorter is walked and each entry found in the
// longer one, by a merge when the lengths are close and by a galloping
// search when one list is much longer.  Per-vertex counts are emitted as
// (vertex, count) pairs, u and v once per in-edge with triangles and w once
// per match, per thread; the caller adds them into the device counters.
//
// It reads a host mirror of the oriented graph (row offsets, columns, row
// of each edge, in-edge offsets and ranges), copied from the device once per
// partition and kept on the blocks handle.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>

#include "hybrid.cuh"

namespace pgb {

namespace {

struct HostMirror {
    uint32_t n = 0;
    uint64_t m = 0;
    std::vector<uint32_t> rowptr, col, rowidx, colptr;
    std::vector<unsigned long long> xr;
};

// first position in a[b, e) whose entry is >= x, searching from b with
// doubling steps (cheap when the answer is near b)
inline uint32_t gallop(const uint32_t* a, uint32_t b, uint32_t e, uint32_t x) {
    uint32_t step = 1, lo = b, hi = b;
    while (hi < e && a[hi] < x) {
        lo = hi + 1;
        hi = (e - hi > step) ? hi + step : e;
        step <<= 1;
    }
    return (uint32_t)(std::lower_bound(a + lo, a + hi, x) - a);
}

// Matches of the sorted ranges col[xb, xe) and col[yb, ye); each common
// entry w calls on_match(w).  Returns the number of matches.
template <class F>
inline uint64_t intersect(const uint32_t* col, uint32_t xb, uint32_t xe, uint32_t yb, uint32_t ye, F&& on_match) {
    uint64_t c = 0;
    uint32_t lx = xe - xb, ly = ye - yb;
    if (!lx || !ly) return 0;
    if (lx > ly) {
        std::swap(xb, yb);
        std::swap(xe, ye);
        std::swap(lx, ly);
    }
    if (ly > 16 * lx) {
        uint32_t q = yb;
        for (uint32_t a = xb; a < xe && q < ye; ++a) {
            q = gallop(col, q, ye, col[a]);
            if (q < ye && col[q] == col[a]) {
                ++c;
                on_match(col[a]);
                ++q;
            }
        }
        return c;
    }
    uint32_t a = xb, q = yb;
    while (a < xe && q < ye) {
        const uint32_t va = col[a], vb = col[q];
        if (va < vb) ++a;
        else if (vb < va) ++q;
        else {
            ++c;
            on_match(va);
            ++a;
            ++q;
        }
    }
    return c;
}

const HostMirror& mirror_of(const pgb_blocks* b, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(b->plan_mu);
    if (!b->host_mirror) {
        auto H = std::make_shared<HostMirror>();
        H->n = b->n;
        H->m = b->m;
        H->rowptr.resize((size_t)b->n + 1);
        H->colptr.resize((size_t)b->n + 1);
        H->col.resize(b->m);
        H->rowidx.resize(b->m);
        H->xr.resize(b->m);
        PGB_CUDA(cudaMemcpyAsync(H->rowptr.data(), b->rowptr.ptr, ((size_t)b->n + 1) * 4, cudaMemcpyDeviceToHost, s));
        PGB_CUDA(cudaMemcpyAsync(H->colptr.data(), b->colptr.ptr, ((size_t)b->n + 1) * 4, cudaMemcpyDeviceToHost, s));
        if (b->m) {
            PGB_CUDA(cudaMemcpyAsync(H->col.data(), b->col.ptr, b->m * 4, cudaMemcpyDeviceToHost, s));
            PGB_CUDA(cudaMemcpyAsync(H->rowidx.data(), b->rowidx.ptr, b->m * 4, cudaMemcpyDeviceToHost, s));
            PGB_CUDA(cudaMemcpyAsync(H->xr.data(), b->xr.ptr, b->m * 8, cudaMemcpyDeviceToHost, s));
        }
        PGB_CUDA(cudaStreamSynchronize(s));
        b->host_mirror = H;
    }
    return *std::static_pointer_cast<HostMirror>(b->host_mirror);
}

}  // namespace

std::vector<uint8_t> host_parts_by_cutoff(const pgb_blocks* b, uint32_t share_ppm) {
    const uint32_t p = b->p;
    std::vector<uint8_t> host(p, 0);
    std::vector<uint64_t> est(p, 0);
    uint64_t total = 0;
    for (uint32_t j = 0; j < p; ++j) {
        const uint64_t in_edges = b->head_off.size() > j + 1 ? b->head_off[j + 1] - b->head_off[j] : 0;
        est[j] = (j < b->part_probes.size() ? b->part_probes[j] : 0) + in_edges;
        total += est[j];
    }
    // lightest first (ties: higher part first, so that the heaviest-ranked
    // heads stay on the device); stop at the first part past the cut-off
    std::vector<uint32_t> order(p);
    for (uint32_t j = 0; j < p; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
        if (est[x] != est[y]) return est[x] < est[y];
        return x > y;
    });
    const long double cap = (long double)total * share_ppm / 1e6L;
    long double acc = 0;
    for (uint32_t j : order) {
        if (est[j] == 0) continue;  // nothing to count
        if (acc + est[j] > cap) break;
        acc += est[j];
        host[j] = 1;
    }
    return host;
}

HostCountResult host_count_parts(const pgb_blocks* b, const std::vector<uint8_t>& host, uint32_t threads,
                                 bool per_vertex, std::vector<std::pair<uint32_t, uint32_t>>& adds,
                                 const pgb_cancel* cancel, cudaStream_t s, uint32_t core_e0) {
    HostCountResult R;
    const auto t0 = std::chrono::steady_clock::now();
    // head runs of the host parts, lightest part first
    std::vector<std::pair<uint32_t, uint32_t>> runs;
    std::vector<uint32_t> parts;
    for (uint32_t j = 0; j < b->p; ++j)
        if (host[j]) parts.push_back(j);
    if (parts.empty()) return R;
    const HostMirror& H = mirror_of(b, s);
    std::stable_sort(parts.begin(), parts.end(), [&](uint32_t x, uint32_t y) {
        return b->part_probes[x] + (b->head_off[x + 1] - b->head_off[x]) <
               b->part_probes[y] + (b->head_off[y + 1] - b->head_off[y]);
    });
    constexpr uint32_t kRun = 256;  // heads per claimed run
    for (uint32_t j : parts) {
        R.in_edges += b->head_off[j + 1] - b->head_off[j];
        for (uint32_t v = b->cuts[j]; v < b->cuts[j + 1]; v += kRun)
            runs.emplace_back(v, std::min(v + kRun, b->cuts[j + 1]));
    }
    R.parts = (uint32_t)parts.size();
    if (threads == 0) threads = std::max(1u, std::thread::hardware_concurrency());
    threads = std::min<uint32_t>(threads, (uint32_t)std::max<size_t>(runs.size(), 1));
    std::atomic<size_t> next{0};
    std::atomic<uint64_t> total{0};
    std::atomic<bool> stopped{false};
    const uint32_t* col = H.col.data();
    std::vector<std::vector<std::pair<uint32_t, uint32_t>>> local(threads);
    auto worker = [&](uint32_t id) {
        uint64_t mine = 0;
        std::vector<std::pair<uint32_t, uint32_t>>& out = local[id];
        for (;;) {
            if (cancel && __atomic_load_n(const_cast<const uint32_t*>(cancel->host), __ATOMIC_RELAXED)) {
                stopped = true;
                break;
            }
            const size_t k = next.fetch_add(1);
            if (k >= runs.size()) break;
            for (uint32_t v = runs[k].first; v < runs[k].second; ++v) {
                const uint32_t vb = H.rowptr[v], ve = H.rowptr[v + 1];
                if (vb == ve) continue;
                uint64_t cv = 0;
                for (uint32_t q = H.colptr[v]; q < H.colptr[v + 1]; ++q) {
                    const unsigned long long r = H.xr[q];
                    const uint32_t xb = (uint32_t)r, xe = (uint32_t)(r >> 32);
                    if (xb - 1 >= core_e0) continue;  // the tail is in the dense top block
                    uint64_t c;
                    if (per_vertex) c = intersect(col, xb, xe, vb, ve, [&](uint32_t w) { out.emplace_back(w, 1u); });
                    else c = intersect(col, xb, xe, vb, ve, [](uint32_t) {});
                    if (c && per_vertex) out.emplace_back(H.rowidx[xb - 1], (uint32_t)c);
                    cv += c;
                }
                // (a head's total may pass 2^32: emitted in pieces of 2^31)
                for (uint64_t left = per_vertex ? cv : 0; left;) {
                    const uint32_t piece = (uint32_t)std::min<uint64_t>(left, 1ull << 31);
                    out.emplace_back(v, piece);
                    left -= piece;
                }
                mine += cv;
            }
        }
        total += mine;
    };
    std::vector<std::thread> pool;
    for (uint32_t k = 1; k < threads; ++k) pool.emplace_back(worker, k);
    worker(0);
    for (auto& th : pool) th.join();
    for (auto& l : local) adds.insert(adds.end(), l.begin(), l.end());
    R.total = total.load();
    R.cancelled = stopped.load();
    R.threads = threads;
    R.ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return R;
}

}  // namespace pgb
