// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "pgabb.h"

namespace pgb {

// ------------------------------------------------------------------ errors

// Thrown inside the library only; every extern "C" entry converts it to a
// status code through guard().
struct Error {
    int code;
    std::string msg;
};

void set_error(const std::string& msg);
[[noreturn]] void fail(int code, const std::string& msg);

#define PGB_CUDA(call)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            ::pgb::fail(e_ == cudaErrorMemoryAllocation ? PGB_E_NOMEM : PGB_E_CUDA,        \
                        std::string(#call) + ": " + cudaGetErrorString(e_));               \
    } while (0)

// Check the launch(es) just issued and count them as the library's own
// kernel launches (library primitives such as CUB sorts are not counted).
#define PGB_CHECK_LAUNCHES(what, k)                                                        \
    do {                                                                                   \
        ::pgb::note_launches(k);                                                           \
        cudaError_t e_ = cudaGetLastError();                                               \
        if (e_ != cudaSuccess)                                                             \
            ::pgb::fail(PGB_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e_));    \
    } while (0)
#define PGB_CHECK_LAUNCH(what) PGB_CHECK_LAUNCHES(what, 1)

void note_launches(uint64_t k);
// While a capture is open in this thread, launches are counted into
// *counter instead (a captured launch runs only when the graph is replayed).
void begin_launch_capture(uint64_t* counter);
void end_launch_capture();

template <class F>
int guard(F&& f) {
    try {
        f();
        return PGB_OK;
    } catch (const Error& e) {
        set_error(e.msg);
        return e.code;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return PGB_E_NOMEM;
    } catch (...) {
        set_error("unexpected internal error");
        return PGB_E_CUDA;
    }
}

// --------------------------------------------------------------- allocator

// dev_alloc reports in *native whether the memory came from the CUDA
// stream-ordered allocator (true) or from the registered hooks (false); the
// matching dev_free needs that flag.
void* dev_alloc(size_t bytes, cudaStream_t s, bool* native);
void dev_free(void* p, size_t bytes, cudaStream_t s, bool native);
// Make the calling thread use the CUDA stream-ordered allocator even when
// hooks are registered (for the library's own threads, which must not call
// back into the host program).
// Device memory of this thread's library calls: stream-ordered allocations
// from `pool` (nullptr: the device's default pool), never the hooks set with
// pgb_set_allocator.
void use_native_allocator_in_this_thread(cudaMemPool_t pool = nullptr);
void live_handles_add(int d);

// Owning device buffer that returns its memory to the library allocator on
// the stream it was allocated on.
template <class T>
struct DevBuf {
    T* ptr = nullptr;
    size_t count = 0;
    cudaStream_t stream = nullptr;
    bool native = false;

    DevBuf() = default;
    DevBuf(size_t n, cudaStream_t s) { alloc(n, s); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept { swap(o); }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) {
            release();
            swap(o);
        }
        return *this;
    }
    ~DevBuf() { release(); }

    void swap(DevBuf& o) noexcept {
        std::swap(ptr, o.ptr);
        std::swap(count, o.count);
        std::swap(stream, o.stream);
        std::swap(native, o.native);
    }
    void alloc(size_t n, cudaStream_t s) {
        release();
        stream = s;
        count = n;
        ptr = n ? static_cast<T*>(dev_alloc(n * sizeof(T), s, &native)) : nullptr;
    }
    void release() {
        if (ptr) dev_free(ptr, count * sizeof(T), stream, native);
        ptr = nullptr;
        count = 0;
    }
    size_t bytes() const { return count * sizeof(T); }
};

// Scratch bytes for library primitives (CUB temp storage).
struct Scratch {
    DevBuf<unsigned char> buf;
    void* get(size_t bytes, cudaStream_t s) {
        if (buf.count < bytes) buf.alloc(bytes + (bytes >> 3) + 256, s);
        return buf.ptr;
    }
};

int num_bits(uint64_t x);  // bits needed to represent values in [0, x]

// ------------------------------------------------------------ stop requests

// Per-run control block in device memory.  `stop` points at the run's
// cancel-token word (pinned host memory mapped into the device's address
// space) or is null; a kernel that sees the word set skips the rest of its
// work and sets `cancelled`.
struct RunCtl {
    const volatile uint32_t* stop;
    uint32_t cancelled;
    uint32_t pad;
};

// The persistent kernels call this once every kStopCheckEvery work fetches
// (a plain per-triple launch once at entry): a rare read of a word in host
// memory, so that a stop request ends a run within a few work items.
constexpr uint32_t kStopCheckEvery = 64;

#ifdef __CUDACC__
__device__ __forceinline__ bool run_stop_requested(RunCtl* c) {
    if (!c) return false;
    const volatile uint32_t* st = *reinterpret_cast<const volatile uint32_t* const volatile*>(&c->stop);
    if (!st || *st == 0u) return false;
    *reinterpret_cast<volatile uint32_t*>(&c->cancelled) = 1u;
    return true;
}
#endif

// ------------------------------------------------------------------ handles

}  // namespace pgb

struct pgb_graph {
    uint32_t n = 0;
    uint64_t m = 0;                       // unique undirected edges
    uint32_t id_bits = 1;                 // bits per packed endpoint
    pgb::DevBuf<uint64_t> keys;           // (a << id_bits) | b, a < b, sorted
    pgb::DevBuf<uint32_t> deg;            // degree per vertex
    cudaStream_t stream = nullptr;
};

// A cancel token: one word of pinned host memory, mapped into the device's
// address space, that the host sets and the kernels read.
struct pgb_cancel {
    volatile uint32_t* host = nullptr;
    uint32_t* dev = nullptr;
};

struct pgb_triple {
    uint32_t i, j, k;
    uint64_t w;
};

struct pgb_blocks {
    uint32_t n = 0, p = 0;
    uint64_t m = 0;
    cudaStream_t stream = nullptr;
    // offloaded in-edge index (pgb_blocks_offload): per in-edge the tail-row
    // range after the head (xr) and the tail, in pinned host memory
    bool offloaded = false;
    unsigned long long* h_xr = nullptr;
    uint32_t* h_itail = nullptr;
    // columns offloaded too (pgb_blocks_offload_columns): slices, the
    // tail-block-major index and the pieces' work items (stream.cu)
    bool cols_offloaded = false;
    std::shared_ptr<void> col_plan;
    // chunking of the last streamed run's settings (stream.cu)
    mutable std::shared_ptr<void> stream_plan;
    // captured runs (use_graph), at most four settings (tc.cu)
    mutable std::vector<std::shared_ptr<void>> run_plans;
    mutable std::mutex plan_mu;
    // host copy of the oriented graph for the hybrid host kernel (hybrid.cu)
    mutable std::shared_ptr<void> host_mirror;
    ~pgb_blocks() {
        if (h_xr) cudaFreeHost(h_xr);
        if (h_itail) cudaFreeHost(h_itail);
    }
    pgb::DevBuf<uint32_t> perm;    // rank -> original ID
    pgb::DevBuf<uint32_t> rowptr;  // n + 1 oriented offsets (m < 2^32)
    pgb::DevBuf<uint32_t> col;     // m oriented columns, rank space, rows sorted
    pgb::DevBuf<uint32_t> rowidx;  // m row of each oriented edge
    // m CSR edge positions grouped by block (i, j) row-major; built on first
    // use by ensure_block_edge_index (guarded by bedge_mu)
    mutable pgb::DevBuf<uint32_t> bedge;
    mutable bool bedge_ready = false;
    mutable std::mutex bedge_mu;
    pgb::DevBuf<uint32_t> colptr;  // n + 1 first in-edge of each head v (in-edge index order)
    pgb::DevBuf<unsigned long long> xr;  // m in-edges grouped by head: tail-row range after v
    pgb::DevBuf<uint32_t> cuts_d;  // p + 1
    std::vector<uint32_t> cuts;    // p + 1
    std::vector<uint64_t> block_edges;  // p * p
    std::vector<uint64_t> block_off;    // p * p + 1 offsets into bedge
    std::vector<pgb_triple> triples;    // queue order
    uint64_t wedges = 0;
    uint64_t probes = 0;  // sum over edges (u, v) of the entries of u's row after v
    std::vector<uint64_t> part_probes;  // p: the same sum over edges whose head v lies in part j
    std::vector<uint64_t> head_off;     // p + 1: first in-edge (index order) of each head part
    // lookups of the in-edges whose tail has rank in [n - 1024 (i + 1), n - 1024 i), i < 32: what a
    // dense top block of 1024 (i + 1) ranks would take from the intersection kernels (core.cu)
    std::vector<uint64_t> core_probes;
    uint32_t max_outdeg = 0;
};

namespace pgb {

// Kernel-side stages (each enqueued on `s`; those that need sizes sync).
void ingest_keys(pgb_graph* g, const uint32_t* src, const uint32_t* dst, uint64_t m, cudaStream_t s);
void build_partition(const pgb_graph* g, uint32_t p, int rule, cudaStream_t s, pgb_blocks* b);
void ensure_block_edge_index(const pgb_blocks* b, cudaStream_t s);
void copy_out(void* dst, const void* src_dev, size_t bytes, int mem, cudaStream_t s);
// Upper block IDs (i * p + j, i <= j) along the Hilbert curve (blocks.cu).
std::vector<uint32_t> hilbert_block_order(uint32_t p);
// Pinned host copy of the columns after pgb_blocks_offload_columns, else null.
const uint32_t* offloaded_columns(const pgb_blocks* b);

}  // namespace pgb
