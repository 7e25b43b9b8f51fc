// Error reporting, the device allocator hook and small shared helpers.
#include <atomic>
#include <mutex>

#include "internal.cuh"

namespace pgb {

static thread_local std::string t_last_error = "";

void set_error(const std::string& msg) { t_last_error = msg; }

void fail(int code, const std::string& msg) { throw Error{code, msg}; }

static std::mutex g_alloc_mu;
static pgb_alloc_fn g_alloc = nullptr;
static pgb_free_fn g_free = nullptr;
static void* g_ctx = nullptr;
static std::atomic<long> g_live{0};
static std::atomic<uint64_t> g_launches{0};

static thread_local uint64_t* t_capture_count = nullptr;

void note_launches(uint64_t k) {
    if (t_capture_count) *t_capture_count += k;
    else g_launches += k;
}

void begin_launch_capture(uint64_t* counter) { t_capture_count = counter; }
void end_launch_capture() { t_capture_count = nullptr; }

void live_handles_add(int d) { g_live += d; }

static thread_local bool t_native_only = false;
static thread_local cudaMemPool_t t_pool = nullptr;

void use_native_allocator_in_this_thread(cudaMemPool_t pool) {
    t_native_only = true;
    t_pool = pool;
}

void* dev_alloc(size_t bytes, cudaStream_t s, bool* native) {
    if (bytes == 0) return nullptr;
    void* p = nullptr;
    if (g_alloc && !t_native_only) {
        *native = false;
        p = g_alloc(bytes, s, g_ctx);
        if (!p) fail(PGB_E_NOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
        if (reinterpret_cast<uintptr_t>(p) & 255) {
            // kernels read rows with aligned 16- and 32-byte loads
            g_free(p, bytes, s, g_ctx);
            fail(PGB_E_INVAL, "the allocator hook returned memory not aligned to 256 bytes");
        }
        return p;
    }
    *native = true;
    cudaError_t e = t_pool ? cudaMallocFromPoolAsync(&p, bytes, t_pool, s) : cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        fail(PGB_E_NOMEM, "cudaMallocAsync of " + std::to_string(bytes) + " bytes failed: " +
                              cudaGetErrorString(e));
    }
    return p;
}

void dev_free(void* p, size_t bytes, cudaStream_t s, bool native) {
    if (!p) return;
    if (!native && g_free) {
        g_free(p, bytes, s, g_ctx);
        return;
    }
    cudaFreeAsync(p, s);
}

int num_bits(uint64_t x) {
    int b = 0;
    while (b < 64 && (x >> b) != 0) ++b;
    return b < 1 ? 1 : b;
}

void copy_out(void* dst, const void* src_dev, size_t bytes, int mem, cudaStream_t s) {
    if (bytes == 0) return;
    if (!dst) fail(PGB_E_INVAL, "NULL destination");
    PGB_CUDA(cudaMemcpyAsync(dst, src_dev, bytes,
                             mem == PGB_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (mem != PGB_MEM_DEVICE) PGB_CUDA(cudaStreamSynchronize(s));
}

}  // namespace pgb

extern "C" {

const char* pgb_last_error(void) { return pgb::t_last_error.c_str(); }

const char* pgb_version(void) { return "pgabb-b300 0.2.0 (sm_103a)"; }

int pgb_cancel_create(pgb_cancel** out) {
    return pgb::guard([&] {
        if (!out) pgb::fail(PGB_E_INVAL, "out is NULL");
        std::unique_ptr<pgb_cancel> c(new pgb_cancel());
        void* h = nullptr;
        PGB_CUDA(cudaHostAlloc(&h, 64, cudaHostAllocMapped | cudaHostAllocPortable));
        std::memset(h, 0, 64);
        void* d = nullptr;
        cudaError_t e = cudaHostGetDevicePointer(&d, h, 0);
        if (e != cudaSuccess) {
            cudaFreeHost(h);
            pgb::fail(PGB_E_CUDA, std::string("cudaHostGetDevicePointer: ") + cudaGetErrorString(e));
        }
        c->host = static_cast<volatile uint32_t*>(h);
        c->dev = static_cast<uint32_t*>(d);
        *out = c.release();
    });
}

int pgb_cancel_set(pgb_cancel* c) {
    return pgb::guard([&] {
        if (!c) pgb::fail(PGB_E_INVAL, "token is NULL");
        __atomic_store_n(const_cast<uint32_t*>(c->host), 1u, __ATOMIC_SEQ_CST);
    });
}

int pgb_cancel_reset(pgb_cancel* c) {
    return pgb::guard([&] {
        if (!c) pgb::fail(PGB_E_INVAL, "token is NULL");
        __atomic_store_n(const_cast<uint32_t*>(c->host), 0u, __ATOMIC_SEQ_CST);
    });
}

int pgb_cancel_is_set(const pgb_cancel* c, int* set) {
    return pgb::guard([&] {
        if (!c || !set) pgb::fail(PGB_E_INVAL, "NULL argument");
        *set = __atomic_load_n(const_cast<const uint32_t*>(c->host), __ATOMIC_SEQ_CST) != 0;
    });
}

void pgb_cancel_free(pgb_cancel* c) {
    if (!c) return;
    if (c->host) cudaFreeHost(const_cast<uint32_t*>(c->host));
    delete c;
}

uint64_t pgb_kernel_launches(void) { return pgb::g_launches.load(); }

int pgb_set_allocator(pgb_alloc_fn alloc, pgb_free_fn free_fn, void* ctx) {
    return pgb::guard([&] {
        if ((alloc == nullptr) != (free_fn == nullptr))
            pgb::fail(PGB_E_INVAL, "alloc and free must both be set or both be NULL");
        std::lock_guard<std::mutex> lk(pgb::g_alloc_mu);
        if (pgb::g_live.load() != 0) pgb::fail(PGB_E_STATE, "allocator changed while handles are alive");
        pgb::g_alloc = alloc;
        pgb::g_free = free_fn;
        pgb::g_ctx = ctx;
    });
}

}  // extern "C"
