// Serve loop: triangle-count jobs on graphs of mixed sizes, admitted by an
// HBM budget and counted with continuous batching.
//
// The paper runs one computation at a time (Section 4.1); this file is the
// serving side of the same block-tuple path.  A job is a raw edge list.
//   submit   copies the edges into the job (the caller's arrays are only
//            borrowed for the call) and queues it: host arrays into host
//            memory, device arrays into a device buffer that the job keeps
//            until its batch copies it; a job that can never fit the budget
//            is refused with PGB_E_BUDGET.
//   batch    each of the server's batch threads takes the queued jobs that
//            fit the budget (in arrival order, up to max_batch_jobs and
//            batch_edges raw edges) and counts them as ONE graph: the
//            disjoint union of the jobs, vertex IDs shifted by the vertex
//            counts of the jobs before them.  One ingest, one degree order,
//            one p x p partition and one persistent counting launch serve
//            the whole batch, so the block tuples of all its jobs interleave
//            in that launch.  Triangles never join two jobs, so a job's
//            per-vertex counts are its slice of the union's, and its total is
//            a third of their sum.  Jobs that arrive while a batch runs go
//            into the next batch a thread takes (continuous batching); with
//            several threads, batches overlap on the device.
//   serial   (SERIAL mode) one thread, one job per batch: the baseline.
// An edge with an endpoint >= its job's n fails that job alone: the union
// builder turns the job's edges into self-loops (dropped by ingest) and flags
// the job.  Results (total, per-vertex counts by original ID, latency from
// submit to completion) are kept in the job until it is waited for.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "internal.cuh"

namespace pgb {

// Union edge list: edge i of job j (eoff[j] <= i < eoff[j+1]) gets the job's
// vertex offset voff[j]; an endpoint >= the job's n flags the job and turns
// the edge into a self-loop.
__global__ void k_union_ids(uint32_t* __restrict__ src, uint32_t* __restrict__ dst, uint64_t m,
                            const uint64_t* __restrict__ eoff, const uint64_t* __restrict__ voff, uint32_t nj,
                            uint32_t* __restrict__ bad) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        uint32_t lo = 0, hi = nj;  // job j: largest j with eoff[j] <= i
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (eoff[mid] <= i) lo = mid; else hi = mid;
        }
        const uint64_t n = voff[lo + 1] - voff[lo];
        uint32_t a = src[i], b = dst[i];
        if (a >= n || b >= n) {
            bad[lo] = 1;
            a = b = 0;
        }
        src[i] = (uint32_t)(voff[lo] + a);
        dst[i] = (uint32_t)(voff[lo] + b);
    }
}

// sums[j] = sum of t over job j's vertex range [voff[j], voff[j+1]).
__global__ void k_job_sums(const unsigned long long* __restrict__ t, const uint64_t* __restrict__ voff,
                           unsigned long long* __restrict__ sums) {
    __shared__ unsigned long long red[32];
    const uint32_t j = blockIdx.x;
    unsigned long long acc = 0;
    for (uint64_t x = voff[j] + threadIdx.x; x < voff[j + 1]; x += blockDim.x) acc += t[x];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) sums[j] = acc;
    }
}

using Clock = std::chrono::steady_clock;

struct Job {
    uint64_t id = 0;
    int state = PGB_JOB_QUEUED;
    int err = PGB_OK;
    std::string msg;
    uint32_t n = 0;
    uint64_t m = 0;
    uint64_t est = 0;  // admitted device bytes
    std::vector<uint32_t> src, dst;
    // device input (src then dst, 8 bytes per raw edge), until the batch
    // copies it; allocated and freed stream-ordered
    void* dmem = nullptr;
    // borrowed input (pgb_server_submit_borrowed): the caller's arrays, in
    // device or host memory
    const uint32_t* bsrc = nullptr;
    const uint32_t* bdst = nullptr;
    Clock::time_point submitted, finished;
    // results
    uint64_t total = 0;
    std::vector<uint64_t> per_vertex;
    bool cancel = false;
    std::shared_ptr<struct BatchState> batch;  // while RUNNING: the batch it is in

    void drop_input(cudaStream_t s) {
        src.clear();
        src.shrink_to_fit();
        dst.clear();
        dst.shrink_to_fit();
        if (dmem) cudaFreeAsync(dmem, s);
        dmem = nullptr;
    }
    ~Job() { drop_input(cudaStreamLegacy); }
};

// A batch on the device: its thread's cancel token and how many of its jobs
// are not cancelled; when that reaches zero the token stops the kernels.
struct BatchState {
    pgb_cancel* token = nullptr;
    size_t live = 0;
};

// Pinned host buffers for batch results, reused by one batch thread.
struct PinnedPool {
    void* ptr = nullptr;
    size_t size = 0;
    void* get(size_t bytes) {
        if (bytes > size) {
            if (ptr) cudaFreeHost(ptr);
            ptr = nullptr;
            size = 0;
            const size_t sz = std::max<size_t>(bytes + bytes / 4, 1 << 20);
            PGB_CUDA(cudaHostAlloc(&ptr, sz, cudaHostAllocDefault));
            size = sz;
        }
        return ptr;
    }
    ~PinnedPool() {
        if (ptr) cudaFreeHost(ptr);
    }
};

// Caps of one batch: raw edges (unless a single job is larger) and vertices.
constexpr uint64_t kDefaultBatchEdges = 1ull << 27;
constexpr uint64_t kMaxBatchVertices = 1ull << 31;
constexpr uint32_t kMaxJobsPerBatch = 4096;

}  // namespace pgb

struct pgb_server {
    pgb_server_opts o{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_queue;   // queued jobs / budget freed / stop
    std::condition_variable cv_done;    // job completions
    std::deque<std::shared_ptr<pgb::Job>> queued;
    std::map<uint64_t, std::shared_ptr<pgb::Job>> jobs;
    uint64_t next_id = 1;
    uint64_t bytes_in_use = 0;
    uint64_t n_done = 0, n_failed = 0, n_cancelled = 0, n_batches = 0, jobs_in_batches = 0;
    bool stop = false;
    bool paused = false;  // admission held (queued jobs wait)
    std::vector<std::thread> threads;
    std::vector<cudaStream_t> streams;  // one per batch thread, for the server's lifetime
    std::vector<pgb_cancel*> tokens;    // one per batch thread: stops its batch's kernels
    // the server's own stream-ordered memory pool: batches and queued device
    // inputs allocate from it, and memory freed there stays mapped for the
    // next batch until the server is destroyed (the device's default pool
    // gives freed memory back at every synchronisation)
    cudaMemPool_t pool = nullptr;
};

namespace pgb {

uint64_t job_bytes(uint64_t m, uint32_t n) {
    // ingest: raw copy 8 + keys and sort buffers 16 + CUB scratch ~16 per raw
    // edge; partition: CSR, row index, ranges and their sort buffers ~40 per
    // edge; per-vertex data ~48 per vertex; plus a fixed 4 MiB of slack
    return 80 * m + 48 * ((uint64_t)n + 1) + (4ull << 20);
}

static void finish(pgb_server* S, const std::shared_ptr<Job>& J, int state, int err, const std::string& msg) {
    std::lock_guard<std::mutex> lk(S->mu);
    J->state = state;
    J->err = err;
    J->msg = msg;
    J->finished = Clock::now();
    J->drop_input(cudaStreamLegacy);
    S->bytes_in_use -= J->est;
    if (state == PGB_JOB_DONE) ++S->n_done;
    else if (state == PGB_JOB_CANCELLED) ++S->n_cancelled;
    else ++S->n_failed;
    S->cv_done.notify_all();
    S->cv_queue.notify_all();
}

// Count one batch as the disjoint union of its jobs (see the top of this
// file); fills each job's total and per-vertex counts, and `bad[j]` for jobs
// with an endpoint >= n.
static void count_batch(pgb_server* S, const std::vector<std::shared_ptr<Job>>& batch, cudaStream_t s,
                        PinnedPool& pool, std::vector<uint32_t>& bad, pgb_cancel* token) {
    const uint32_t nj = (uint32_t)batch.size();
    std::vector<uint64_t> eoff(nj + 1, 0), voff(nj + 1, 0);
    for (uint32_t j = 0; j < nj; ++j) {
        eoff[j + 1] = eoff[j] + batch[j]->m;
        voff[j + 1] = voff[j] + batch[j]->n;
    }
    const uint64_t M = eoff[nj], N = voff[nj];
    if (N >= kMaxBatchVertices) fail(PGB_E_OVERFLOW, "batch has too many vertices");
    DevBuf<uint64_t> deoff(nj + 1, s), dvoff(nj + 1, s);
    DevBuf<uint32_t> dbad(nj, s);
    PGB_CUDA(cudaMemcpyAsync(deoff.ptr, eoff.data(), (nj + 1) * 8, cudaMemcpyHostToDevice, s));
    PGB_CUDA(cudaMemcpyAsync(dvoff.ptr, voff.data(), (nj + 1) * 8, cudaMemcpyHostToDevice, s));
    PGB_CUDA(cudaMemsetAsync(dbad.ptr, 0, nj * 4, s));
    pgb_graph* g = nullptr;
    {
        DevBuf<uint32_t> ds(M, s), dd(M, s);
        for (uint32_t j = 0; j < nj; ++j) {
            Job& J = *batch[j];
            if (!J.m) continue;
            if (J.bsrc) {
                // borrowed arrays in device or (ideally pinned) host memory
                PGB_CUDA(cudaMemcpyAsync(ds.ptr + eoff[j], J.bsrc, J.m * 4, cudaMemcpyDefault, s));
                PGB_CUDA(cudaMemcpyAsync(dd.ptr + eoff[j], J.bdst, J.m * 4, cudaMemcpyDefault, s));
            } else if (J.dmem) {
                const uint32_t* in = static_cast<const uint32_t*>(J.dmem);
                PGB_CUDA(cudaMemcpyAsync(ds.ptr + eoff[j], in, J.m * 4, cudaMemcpyDeviceToDevice, s));
                PGB_CUDA(cudaMemcpyAsync(dd.ptr + eoff[j], in + J.m, J.m * 4, cudaMemcpyDeviceToDevice, s));
                PGB_CUDA(cudaFreeAsync(J.dmem, s));
                J.dmem = nullptr;
            } else {
                PGB_CUDA(cudaMemcpyAsync(ds.ptr + eoff[j], J.src.data(), J.m * 4, cudaMemcpyHostToDevice, s));
                PGB_CUDA(cudaMemcpyAsync(dd.ptr + eoff[j], J.dst.data(), J.m * 4, cudaMemcpyHostToDevice, s));
            }
        }
        if (M) {
            k_union_ids<<<(unsigned)std::min<uint64_t>((M + 255) / 256, 148ull * 32), 256, 0, s>>>(
                ds.ptr, dd.ptr, M, deoff.ptr, dvoff.ptr, nj, dbad.ptr);
            PGB_CHECK_LAUNCH("k_union_ids");
        }
        const int rc = pgb_graph_from_edges(ds.ptr, dd.ptr, M, (uint32_t)N, PGB_MEM_DEVICE, s, &g);
        if (rc != PGB_OK) fail(rc, pgb_last_error());
    }
    pgb_blocks* b = nullptr;
    const uint32_t p = N ? (uint32_t)std::min<uint64_t>(S->o.p ? S->o.p : 8, N) : 1;
    int rc = pgb_partition(g, p, PGB_CUT_NNZ, s, &b);
    pgb_graph_free(g);
    if (rc != PGB_OK) fail(rc, pgb_last_error());
    std::unique_ptr<pgb_blocks, void (*)(pgb_blocks*)> bguard(b, pgb_blocks_free);
    // per-vertex counts are needed even for totals alone: a job's total is a
    // third of the sum over its vertices
    pgb_tc_opts o;
    pgb_tc_opts_default(&o);
    o.cancel = token;
    int stopped = 0;
    pgb_cancel_is_set(token, &stopped);
    if (stopped) fail(PGB_E_CANCELLED, "every job of the batch was cancelled");
    pgb_tc_result* r = nullptr;
    rc = pgb_tc_run(b, &o, s, &r);
    if (rc != PGB_OK) fail(rc, pgb_last_error());
    std::unique_ptr<pgb_tc_result, void (*)(pgb_tc_result*)> rguard(r, pgb_tc_result_free);
    DevBuf<unsigned long long> t(std::max<uint64_t>(N, 1), s), sums(nj, s);
    rc = pgb_tc_result_get(r, nullptr, N ? reinterpret_cast<uint64_t*>(t.ptr) : nullptr, PGB_MEM_DEVICE);
    if (rc != PGB_OK) fail(rc, pgb_last_error());
    k_job_sums<<<nj, 256, 0, s>>>(t.ptr, dvoff.ptr, sums.ptr);
    PGB_CHECK_LAUNCH("k_job_sums");
    // one copy back: sums, flags, then (per-vertex runs) the union's counts
    const bool pv = S->o.per_vertex != 0;
    const size_t head = (size_t)nj * 8 + (size_t)nj * 4;
    unsigned char* h = static_cast<unsigned char*>(pool.get(head + (pv ? N * 8 : 0)));
    PGB_CUDA(cudaMemcpyAsync(h, sums.ptr, nj * 8, cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaMemcpyAsync(h + nj * 8, dbad.ptr, nj * 4, cudaMemcpyDeviceToHost, s));
    if (pv && N) PGB_CUDA(cudaMemcpyAsync(h + head, t.ptr, N * 8, cudaMemcpyDeviceToHost, s));
    PGB_CUDA(cudaStreamSynchronize(s));
    const uint64_t* hs = reinterpret_cast<const uint64_t*>(h);
    const uint32_t* hb = reinterpret_cast<const uint32_t*>(h + nj * 8);
    const uint64_t* ht = reinterpret_cast<const uint64_t*>(h + head);
    bad.assign(hb, hb + nj);
    for (uint32_t j = 0; j < nj; ++j) {
        Job& J = *batch[j];
        J.total = hs[j] / 3;
        if (pv) J.per_vertex.assign(ht + voff[j], ht + voff[j + 1]);
    }
}

static void batch_loop(pgb_server* S, int idx) {
    cudaSetDevice(S->device);
    use_native_allocator_in_this_thread(S->pool);
    const cudaStream_t s = S->streams[idx];
    const bool serial = S->o.mode == PGB_SERVE_SERIAL;
    const uint32_t cap = serial ? 1 : (S->o.max_batch_jobs ? S->o.max_batch_jobs : 256);
    const uint64_t max_edges = S->o.batch_edges ? S->o.batch_edges : kDefaultBatchEdges;
    PinnedPool pool;
    pgb_cancel* token = S->tokens[idx];
    for (;;) {
        std::vector<std::shared_ptr<Job>> batch;
        std::shared_ptr<BatchState> bs;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_queue.wait(lk, [&] {
                if (S->stop) return true;
                if (S->paused || S->queued.empty()) return false;
                return S->bytes_in_use + S->queued.front()->est <= S->o.budget_bytes;
            });
            if (S->stop) break;
            // the token is reset under the lock, before any job of this batch
            // can be cancelled
            pgb_cancel_reset(token);
            bs = std::make_shared<BatchState>();
            bs->token = token;
            // admit in arrival order while the budget and the batch caps allow
            uint64_t edges = 0, verts = 0;
            while (!S->queued.empty() && batch.size() < cap) {
                const std::shared_ptr<Job>& J = S->queued.front();
                if (S->bytes_in_use + J->est > S->o.budget_bytes) break;
                if (!batch.empty() && (edges + J->m > max_edges || verts + J->n >= kMaxBatchVertices)) break;
                edges += J->m;
                verts += J->n;
                S->bytes_in_use += J->est;
                J->state = PGB_JOB_RUNNING;
                J->batch = bs;
                batch.push_back(J);
                S->queued.pop_front();
            }
            bs->live = batch.size();
            ++S->n_batches;
            S->jobs_in_batches += batch.size();
        }
        std::vector<uint32_t> bad;
        const int rc = guard([&] { count_batch(S, batch, s, pool, bad, token); });
        const std::string msg = rc == PGB_OK ? std::string() : std::string(pgb_last_error());
        for (size_t j = 0; j < batch.size(); ++j) {
            const std::shared_ptr<Job>& J = batch[j];
            J->batch.reset();
            if (rc == PGB_E_CANCELLED) finish(S, J, PGB_JOB_CANCELLED, PGB_E_CANCELLED, "");
            else if (rc != PGB_OK) finish(S, J, PGB_JOB_FAILED, rc, msg);
            else if (bad[j]) finish(S, J, PGB_JOB_FAILED, PGB_E_INVAL, "vertex ID >= n in the job's edges");
            else if (J->cancel) finish(S, J, PGB_JOB_CANCELLED, PGB_E_CANCELLED, "");
            else finish(S, J, PGB_JOB_DONE, PGB_OK, "");
        }
    }
}

}  // namespace pgb

using namespace pgb;

extern "C" {

void pgb_server_opts_default(pgb_server_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->budget_bytes = 64ull << 30;
    o->max_inflight = 1;
    o->p = 8;
    o->mode = PGB_SERVE_BATCHED;
    o->per_vertex = 1;
    o->max_batch_jobs = 256;
}

uint64_t pgb_server_job_bytes(uint64_t m, uint32_t n) { return job_bytes(m, n); }

int pgb_server_create(const pgb_server_opts* opts, pgb_server** out) {
    return guard([&] {
        if (!out) fail(PGB_E_INVAL, "out is NULL");
        std::unique_ptr<pgb_server> S(new pgb_server());
        if (opts) S->o = *opts; else pgb_server_opts_default(&S->o);
        if (S->o.mode != PGB_SERVE_BATCHED && S->o.mode != PGB_SERVE_SERIAL) fail(PGB_E_INVAL, "bad serve mode");
        if (S->o.budget_bytes == 0) S->o.budget_bytes = 64ull << 30;
        if (S->o.max_inflight == 0) S->o.max_inflight = 1;
        if (S->o.max_batch_jobs > kMaxJobsPerBatch) fail(PGB_E_INVAL, "max_batch_jobs must be at most 4096");
        PGB_CUDA(cudaGetDevice(&S->device));
        pgb_server* raw = S.get();
        const int nthreads = S->o.mode == PGB_SERVE_SERIAL ? 1 : (int)std::min<uint32_t>(S->o.max_inflight, 16);
        auto release = [&] {
            for (cudaStream_t x : S->streams) cudaStreamDestroy(x);
            for (pgb_cancel* c : S->tokens) pgb_cancel_free(c);
            if (S->pool) cudaMemPoolDestroy(S->pool);
        };
        {
            cudaMemPoolProps props{};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = S->device;
            PGB_CUDA(cudaMemPoolCreate(&S->pool, &props));
            uint64_t keep = ~0ull;
            cudaError_t e = cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
            if (e != cudaSuccess) {
                release();
                fail(PGB_E_CUDA, std::string("cudaMemPoolSetAttribute: ") + cudaGetErrorString(e));
            }
        }
        for (int i = 0; i < nthreads; ++i) {
            cudaStream_t st = nullptr;
            cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
            if (e != cudaSuccess) {
                release();
                fail(PGB_E_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
            }
            S->streams.push_back(st);
            pgb_cancel* c = nullptr;
            if (pgb_cancel_create(&c) != PGB_OK) {
                const std::string why = pgb_last_error();
                release();
                fail(PGB_E_CUDA, why);
            }
            S->tokens.push_back(c);
        }
        for (int i = 0; i < nthreads; ++i) raw->threads.emplace_back(batch_loop, raw, i);
        live_handles_add(1);
        *out = S.release();
    });
}

// A new job of m raw edges on n vertices, checked against the budget.
static std::shared_ptr<Job> new_job(pgb_server* S, const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n,
                                    uint64_t* job_id) {
    if (!S || !job_id) fail(PGB_E_INVAL, "NULL argument");
    if (m > 0 && (!src || !dst)) fail(PGB_E_INVAL, "src/dst NULL with m > 0");
    if (m > 0 && n == 0) fail(PGB_E_INVAL, "edges given for an empty vertex set");
    auto J = std::make_shared<Job>();
    J->n = n;
    J->m = m;
    J->est = job_bytes(m, n);
    if (J->est > S->o.budget_bytes)
        fail(PGB_E_BUDGET, "job needs about " + std::to_string(J->est) + " device bytes; budget is " +
                               std::to_string(S->o.budget_bytes));
    return J;
}

static void enqueue(pgb_server* S, const std::shared_ptr<Job>& J, uint64_t* job_id) {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) fail(PGB_E_STATE, "server is shutting down");
    J->id = S->next_id++;
    J->submitted = Clock::now();
    S->jobs[J->id] = J;
    S->queued.push_back(J);
    S->cv_queue.notify_all();
    *job_id = J->id;
}

int pgb_server_submit(pgb_server* S, const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n, int mem,
                      uint64_t* job_id) {
    return guard([&] {
        if (mem != PGB_MEM_HOST && mem != PGB_MEM_DEVICE) fail(PGB_E_INVAL, "bad mem kind");
        auto J = new_job(S, src, dst, m, n, job_id);
        if (m) {
            if (mem == PGB_MEM_HOST) {
                J->src.assign(src, src + m);
                J->dst.assign(dst, dst + m);
            } else {
                // on the legacy default stream: after the work the caller
                // queued there (and on other blocking streams)
                PGB_CUDA(cudaMallocFromPoolAsync(&J->dmem, m * 8, S->pool, cudaStreamLegacy));
                uint32_t* in = static_cast<uint32_t*>(J->dmem);
                PGB_CUDA(cudaMemcpyAsync(in, src, m * 4, cudaMemcpyDeviceToDevice, cudaStreamLegacy));
                PGB_CUDA(cudaMemcpyAsync(in + m, dst, m * 4, cudaMemcpyDeviceToDevice, cudaStreamLegacy));
                PGB_CUDA(cudaStreamSynchronize(cudaStreamLegacy));
            }
        }
        enqueue(S, J, job_id);
    });
}

int pgb_server_submit_borrowed(pgb_server* S, const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n,
                               int mem, uint64_t* job_id) {
    return guard([&] {
        if (mem != PGB_MEM_HOST && mem != PGB_MEM_DEVICE) fail(PGB_E_INVAL, "bad mem kind");
        auto J = new_job(S, src, dst, m, n, job_id);
        J->bsrc = m ? src : nullptr;
        J->bdst = m ? dst : nullptr;
        enqueue(S, J, job_id);
    });
}

int pgb_server_pause(pgb_server* S, int paused) {
    return guard([&] {
        if (!S) fail(PGB_E_INVAL, "server is NULL");
        std::lock_guard<std::mutex> lk(S->mu);
        S->paused = paused != 0;
        S->cv_queue.notify_all();
    });
}

int pgb_server_poll(pgb_server* S, uint64_t job_id, int* state) {
    return guard([&] {
        if (!S || !state) fail(PGB_E_INVAL, "NULL argument");
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->jobs.find(job_id);
        if (it == S->jobs.end()) fail(PGB_E_INVAL, "unknown job id");
        *state = it->second->state;
    });
}

int pgb_server_wait(pgb_server* S, uint64_t job_id, double timeout_s, uint64_t* total, uint64_t* per_vertex,
                    double* latency_s) {
    std::shared_ptr<Job> J;
    int rc = guard([&] {
        if (!S) fail(PGB_E_INVAL, "server is NULL");
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->jobs.find(job_id);
        if (it == S->jobs.end()) fail(PGB_E_INVAL, "unknown job id");
        J = it->second;
        auto terminal = [&] { return J->state != PGB_JOB_QUEUED && J->state != PGB_JOB_RUNNING; };
        if (timeout_s < 0) {
            S->cv_done.wait(lk, terminal);
        } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), terminal)) {
            fail(PGB_E_TIMEOUT, "job " + std::to_string(job_id) + " not finished within the timeout");
        }
        // a job waited for to its end is forgotten, whatever the outcome
        S->jobs.erase(it);
        if (J->state == PGB_JOB_CANCELLED) fail(PGB_E_CANCELLED, "job was cancelled");
        if (J->state == PGB_JOB_FAILED) fail(J->err, J->msg);
        if (total) *total = J->total;
        if (per_vertex) {
            if (!S->o.per_vertex) fail(PGB_E_STATE, "server runs without per-vertex counts");
            std::copy(J->per_vertex.begin(), J->per_vertex.end(), per_vertex);
        }
        if (latency_s) *latency_s = std::chrono::duration<double>(J->finished - J->submitted).count();
    });
    return rc;
}

int pgb_server_cancel(pgb_server* S, uint64_t job_id) {
    std::shared_ptr<Job> J;
    int rc = guard([&] {
        if (!S) fail(PGB_E_INVAL, "server is NULL");
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->jobs.find(job_id);
        if (it == S->jobs.end()) fail(PGB_E_INVAL, "unknown job id");
        J = it->second;
        if (J->state == PGB_JOB_RUNNING && J->batch && !J->cancel) {
            // the last job of a running batch to be cancelled stops its kernels
            if (--J->batch->live == 0) pgb_cancel_set(J->batch->token);
        }
        J->cancel = true;
        auto q = std::find(S->queued.begin(), S->queued.end(), J);
        if (q != S->queued.end()) {
            S->queued.erase(q);
            J->state = PGB_JOB_CANCELLED;
            J->err = PGB_E_CANCELLED;
            J->finished = Clock::now();
            J->drop_input(cudaStreamLegacy);
            ++S->n_cancelled;
            S->cv_done.notify_all();
        }
        // a job already on the device: its batch stops once all its jobs
        // are cancelled; otherwise the batch runs on and this result is dropped
    });
    return rc;
}

int pgb_server_stats(pgb_server* S, pgb_server_info* out) {
    return guard([&] {
        if (!S || !out) fail(PGB_E_INVAL, "NULL argument");
        std::lock_guard<std::mutex> lk(S->mu);
        std::memset(out, 0, sizeof(*out));
        out->submitted = S->next_id - 1;
        out->done = S->n_done;
        out->failed = S->n_failed;
        out->cancelled = S->n_cancelled;
        out->queued = S->queued.size();
        out->batches = S->n_batches;
        out->jobs_in_batches = S->jobs_in_batches;
        out->bytes_in_use = S->bytes_in_use;
    });
}

void pgb_server_destroy(pgb_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        for (auto& J : S->queued) {
            J->state = PGB_JOB_CANCELLED;
            J->err = PGB_E_CANCELLED;
            J->drop_input(cudaStreamLegacy);
        }
        S->queued.clear();
        // batches on the device stop at their next check
        for (pgb_cancel* c : S->tokens) pgb_cancel_set(c);
        S->cv_queue.notify_all();
        S->cv_done.notify_all();
    }
    for (auto& t : S->threads) t.join();
    S->jobs.clear();
    for (cudaStream_t st : S->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (pgb_cancel* c : S->tokens) pgb_cancel_free(c);
    // every allocation from the pool has been freed (stream-ordered) by now;
    // its memory goes back once those frees complete
    cudaStreamSynchronize(cudaStreamLegacy);
    cudaMemPoolDestroy(S->pool);
    delete S;
    live_handles_add(-1);
}

}  // extern "C"
