// Serve loop: triangle-count jobs on graphs of mixed sizes, admitted by an
// HBM budget and counted with continuous batching.
//
// The paper runs one computation at a time (Section 4.1); this file is the
// serving side of the same block-tuple path.  A job is a raw edge list.
//   submit     copies the edges into the job (the caller's arrays are only
//              borrowed for the call) and queues it; a job that can never
//              fit the budget is refused with PGB_E_BUDGET.
//   stage      one of `max_inflight` stage threads admits queued jobs while
//              the estimated device bytes of admitted jobs stay within the
//              budget, and on its own stream copies the edges to the device,
//              ingests, orders, partitions and builds the job's work items.
//              Stages of several jobs, and the counting launch below, run at
//              the same time on the device.
//   batch      (BATCHED mode) the batcher thread takes every staged job (up
//              to max_batch_jobs) and counts them all in ONE persistent
//              launch whose work items interleave the jobs' block tuples;
//              jobs staged while it runs go into the next launch.
//   serial     (SERIAL mode) one stage thread stages and counts each job
//              alone, one job at a time: the baseline.
// Results (total, per-vertex counts by original ID, latency from submit to
// completion) are kept in the job until it is waited for.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "internal.cuh"
#include "tc_hash.cuh"

namespace pgb {

__global__ void k_set_job(VItem* __restrict__ items, uint32_t n, uint32_t job) {
    uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) items[i].job = job;
}

__global__ void k_job_totals(const unsigned long long* __restrict__ partials, uint32_t grid,
                             unsigned long long* __restrict__ totals) {
    __shared__ unsigned long long red[32];
    const uint32_t j = blockIdx.x;
    unsigned long long acc = 0;
    for (uint32_t i = threadIdx.x; i < grid; i += blockDim.x) acc += partials[(size_t)j * grid + i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) totals[j] = acc;
    }
}

__global__ void k_job_scatter(const unsigned long long* __restrict__ tv, const uint32_t* __restrict__ perm, uint32_t n,
                              unsigned long long* __restrict__ out) {
    uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) out[perm[r]] = tv[r];
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
    Clock::time_point submitted, finished;
    // staged device state
    pgb_graph* g = nullptr;
    pgb_blocks* b = nullptr;
    DevBuf<VItem> items;
    uint32_t nitems = 0;
    DevBuf<unsigned long long> tv;  // per-vertex counts by rank
    // results
    uint64_t total = 0;
    std::vector<uint64_t> per_vertex;
    bool cancel = false;

    void release_device() {
        items.release();
        tv.release();
        if (b) pgb_blocks_free(b);
        if (g) pgb_graph_free(g);
        b = nullptr;
        g = nullptr;
    }
};

}  // namespace pgb

struct pgb_server {
    pgb_server_opts o{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_queue;   // queued jobs / budget freed / stop
    std::condition_variable cv_ready;   // staged jobs for the batcher / stop
    std::condition_variable cv_done;    // job completions
    std::deque<std::shared_ptr<pgb::Job>> queued;
    std::deque<std::shared_ptr<pgb::Job>> ready;
    std::map<uint64_t, std::shared_ptr<pgb::Job>> jobs;
    uint64_t next_id = 1;
    uint64_t bytes_in_use = 0;
    uint64_t n_done = 0, n_failed = 0, n_cancelled = 0, n_batches = 0, jobs_in_batches = 0;
    bool stop = false;
    bool paused = false;  // admission held (queued jobs wait)
    std::vector<std::thread> threads;
    // streams live as long as the server: job buffers allocated on a stage
    // stream may be released later by the batcher
    std::vector<cudaStream_t> streams;
};

namespace pgb {

uint64_t job_bytes(uint64_t m, uint32_t n) {
    // ingest: raw copy 8 + keys and sort buffers 16 + CUB scratch ~16 per raw
    // edge; partition: CSR, row index, ranges and their sort buffers ~40 per
    // edge; per-vertex data ~48 per vertex; plus a fixed 4 MiB of slack
    return 80 * m + 48 * ((uint64_t)n + 1) + (4ull << 20);
}

static void finish(pgb_server* S, const std::shared_ptr<Job>& J, int state, int err, const std::string& msg) {
    J->release_device();
    std::lock_guard<std::mutex> lk(S->mu);
    J->state = state;
    J->err = err;
    J->msg = msg;
    J->finished = Clock::now();
    J->src.clear();
    J->src.shrink_to_fit();
    J->dst.clear();
    J->dst.shrink_to_fit();
    S->bytes_in_use -= J->est;
    if (state == PGB_JOB_DONE) ++S->n_done;
    else if (state == PGB_JOB_CANCELLED) ++S->n_cancelled;
    else ++S->n_failed;
    S->cv_done.notify_all();
    S->cv_queue.notify_all();
}

// Copy to the device, ingest, order, partition, build work items.
static void stage_job(pgb_server* S, Job& J, cudaStream_t s) {
    DevBuf<uint32_t> ds(J.m, s), dd(J.m, s);
    if (J.m) {
        PGB_CUDA(cudaMemcpyAsync(ds.ptr, J.src.data(), J.m * 4, cudaMemcpyHostToDevice, s));
        PGB_CUDA(cudaMemcpyAsync(dd.ptr, J.dst.data(), J.m * 4, cudaMemcpyHostToDevice, s));
    }
    int rc = pgb_graph_from_edges(ds.ptr, dd.ptr, J.m, J.n, PGB_MEM_DEVICE, s, &J.g);
    if (rc != PGB_OK) fail(rc, pgb_last_error());
    ds.release();
    dd.release();
    uint32_t p = S->o.p ? S->o.p : 8;
    if (J.n > 0) p = std::min<uint32_t>(p, J.n);
    rc = pgb_partition(J.g, p, PGB_CUT_NNZ, s, &J.b);
    if (rc != PGB_OK) fail(rc, pgb_last_error());
    pgb_graph_free(J.g);
    J.g = nullptr;
    J.nitems = build_hash_items(J.b, 0, 0, s, J.items);
    if (S->o.per_vertex) {
        J.tv.alloc(J.n, s);
        if (J.n) PGB_CUDA(cudaMemsetAsync(J.tv.ptr, 0, (size_t)J.n * 8, s));
    }
    PGB_CUDA(cudaStreamSynchronize(s));
}

// Count the staged jobs in one persistent launch on stream s, then fetch
// their totals and per-vertex counts.
static void count_jobs(pgb_server* S, std::vector<std::shared_ptr<Job>>& batch, cudaStream_t s) {
    const uint32_t nj = (uint32_t)batch.size();
    const bool pv = S->o.per_vertex != 0;
    uint64_t total_items = 0;
    for (auto& J : batch) total_items += J->nitems;
    if (total_items >= (1ull << 32)) fail(PGB_E_OVERFLOW, "too many work items in one batch");
    std::vector<HashGraph> hg(nj);
    for (uint32_t j = 0; j < nj; ++j) {
        const pgb_blocks* b = batch[j]->b;
        hg[j] = HashGraph{b->rowptr.ptr, b->col.ptr, b->rowidx.ptr, b->colptr.ptr, b->xr.ptr,
                          pv ? batch[j]->tv.ptr : nullptr, b->n};
    }
    DevBuf<HashGraph> dg(nj, s);
    PGB_CUDA(cudaMemcpyAsync(dg.ptr, hg.data(), nj * sizeof(HashGraph), cudaMemcpyHostToDevice, s));
    DevBuf<VItem> items(std::max<uint64_t>(total_items, 1), s);
    uint64_t off = 0;
    for (uint32_t j = 0; j < nj; ++j) {
        const uint32_t k = batch[j]->nitems;
        if (!k) continue;
        PGB_CUDA(cudaMemcpyAsync(items.ptr + off, batch[j]->items.ptr, (size_t)k * sizeof(VItem),
                                 cudaMemcpyDeviceToDevice, s));
        k_set_job<<<std::min<uint32_t>((k + 255) / 256, 1024), 256, 0, s>>>(items.ptr + off, k, j);
        PGB_CHECK_LAUNCH("k_set_job");
        off += k;
    }
    const int grid = hash_grid(pv);
    DevBuf<unsigned long long> partials((size_t)nj * grid, s), totals(nj, s);
    DevBuf<unsigned int> cursor(1, s);
    if (total_items) {
        launch_hash(dg.ptr, nj, items.ptr, (uint32_t)total_items, pv, s, cursor.ptr, partials.ptr, grid);
        k_job_totals<<<nj, 256, 0, s>>>(partials.ptr, (uint32_t)grid, totals.ptr);
        PGB_CHECK_LAUNCH("k_job_totals");
    } else {
        PGB_CUDA(cudaMemsetAsync(totals.ptr, 0, nj * 8, s));
    }
    std::vector<unsigned long long> ht(nj);
    PGB_CUDA(cudaMemcpyAsync(ht.data(), totals.ptr, nj * 8, cudaMemcpyDeviceToHost, s));
    std::vector<DevBuf<unsigned long long>> outs(nj);
    for (uint32_t j = 0; j < nj; ++j) {
        Job& J = *batch[j];
        J.total = 0;
        if (pv && J.n) {
            outs[j].alloc(J.n, s);
            k_job_scatter<<<std::min<uint32_t>((J.n + 255) / 256, 4096), 256, 0, s>>>(J.tv.ptr, J.b->perm.ptr, J.n,
                                                                                    outs[j].ptr);
            PGB_CHECK_LAUNCH("k_job_scatter");
            J.per_vertex.assign(J.n, 0);
            PGB_CUDA(cudaMemcpyAsync(J.per_vertex.data(), outs[j].ptr, (size_t)J.n * 8, cudaMemcpyDeviceToHost, s));
        }
    }
    PGB_CUDA(cudaStreamSynchronize(s));
    for (uint32_t j = 0; j < nj; ++j) batch[j]->total = ht[j];
}

static void stage_loop(pgb_server* S, int idx) {
    cudaSetDevice(S->device);
    use_native_allocator_in_this_thread();
    cudaStream_t s = S->streams[idx];
    const bool serial = S->o.mode == PGB_SERVE_SERIAL;
    for (;;) {
        std::shared_ptr<Job> J;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_queue.wait(lk, [&] {
                if (S->stop) return true;
                if (S->paused || S->queued.empty()) return false;
                // admit in arrival order while the budget allows
                return S->bytes_in_use + S->queued.front()->est <= S->o.budget_bytes;
            });
            if (S->stop) break;
            J = S->queued.front();
            S->queued.pop_front();
            S->bytes_in_use += J->est;
            J->state = PGB_JOB_RUNNING;
        }
        int rc = guard([&] {
            stage_job(S, *J, s);
            if (serial) {
                std::vector<std::shared_ptr<Job>> one{J};
                count_jobs(S, one, s);
            }
        });
        if (rc != PGB_OK) {
            finish(S, J, PGB_JOB_FAILED, rc, pgb_last_error());
            continue;
        }
        if (serial) {
            finish(S, J, J->cancel ? PGB_JOB_CANCELLED : PGB_JOB_DONE, J->cancel ? PGB_E_CANCELLED : PGB_OK, "");
        } else {
            std::lock_guard<std::mutex> lk(S->mu);
            S->ready.push_back(J);
            S->cv_ready.notify_all();
        }
    }
}

static void batch_loop(pgb_server* S) {
    cudaSetDevice(S->device);
    use_native_allocator_in_this_thread();
    cudaStream_t s = S->streams.back();
    const uint32_t cap = std::min<uint32_t>(S->o.max_batch_jobs ? S->o.max_batch_jobs : 64, kMaxBatchJobs);
    for (;;) {
        std::vector<std::shared_ptr<Job>> batch;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_ready.wait(lk, [&] { return S->stop || !S->ready.empty(); });
            if (S->stop && S->ready.empty()) break;
            while (!S->ready.empty() && batch.size() < cap) {
                batch.push_back(S->ready.front());
                S->ready.pop_front();
            }
            ++S->n_batches;
            S->jobs_in_batches += batch.size();
        }
        int rc = guard([&] { count_jobs(S, batch, s); });
        for (auto& J : batch) {
            if (rc != PGB_OK) finish(S, J, PGB_JOB_FAILED, rc, pgb_last_error());
            else finish(S, J, J->cancel ? PGB_JOB_CANCELLED : PGB_JOB_DONE, J->cancel ? PGB_E_CANCELLED : PGB_OK, "");
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
    o->max_inflight = 8;
    o->p = 8;
    o->mode = PGB_SERVE_BATCHED;
    o->per_vertex = 1;
    o->max_batch_jobs = 64;
}

uint64_t pgb_server_job_bytes(uint64_t m, uint32_t n) { return job_bytes(m, n); }

int pgb_server_create(const pgb_server_opts* opts, pgb_server** out) {
    return guard([&] {
        if (!out) fail(PGB_E_INVAL, "out is NULL");
        std::unique_ptr<pgb_server> S(new pgb_server());
        if (opts) S->o = *opts; else pgb_server_opts_default(&S->o);
        if (S->o.mode != PGB_SERVE_BATCHED && S->o.mode != PGB_SERVE_SERIAL) fail(PGB_E_INVAL, "bad serve mode");
        if (S->o.budget_bytes == 0) S->o.budget_bytes = 64ull << 30;
        if (S->o.max_inflight == 0) S->o.max_inflight = 8;
        if (S->o.max_batch_jobs > kMaxBatchJobs) fail(PGB_E_INVAL, "max_batch_jobs must be at most 256");
        PGB_CUDA(cudaGetDevice(&S->device));
        pgb_server* raw = S.get();
        const int nstage = S->o.mode == PGB_SERVE_SERIAL ? 1 : (int)S->o.max_inflight;
        const int nstreams = nstage + (S->o.mode == PGB_SERVE_BATCHED ? 1 : 0);
        for (int i = 0; i < nstreams; ++i) {
            cudaStream_t st = nullptr;
            cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
            if (e != cudaSuccess) {
                for (cudaStream_t x : S->streams) cudaStreamDestroy(x);
                fail(PGB_E_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
            }
            S->streams.push_back(st);
        }
        for (int i = 0; i < nstage; ++i) raw->threads.emplace_back(stage_loop, raw, i);
        if (S->o.mode == PGB_SERVE_BATCHED) raw->threads.emplace_back(batch_loop, raw);
        live_handles_add(1);
        *out = S.release();
    });
}

int pgb_server_submit(pgb_server* S, const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n, int mem,
                      uint64_t* job_id) {
    return guard([&] {
        if (!S || !job_id) fail(PGB_E_INVAL, "NULL argument");
        if (m > 0 && (!src || !dst)) fail(PGB_E_INVAL, "src/dst NULL with m > 0");
        if (mem != PGB_MEM_HOST && mem != PGB_MEM_DEVICE) fail(PGB_E_INVAL, "bad mem kind");
        if (m > 0 && n == 0) fail(PGB_E_INVAL, "edges given for an empty vertex set");
        auto J = std::make_shared<Job>();
        J->n = n;
        J->m = m;
        J->est = job_bytes(m, n);
        if (J->est > S->o.budget_bytes)
            fail(PGB_E_BUDGET, "job needs about " + std::to_string(J->est) + " device bytes; budget is " +
                                   std::to_string(S->o.budget_bytes));
        J->src.resize(m);
        J->dst.resize(m);
        if (m) {
            if (mem == PGB_MEM_HOST) {
                std::memcpy(J->src.data(), src, m * 4);
                std::memcpy(J->dst.data(), dst, m * 4);
            } else {
                PGB_CUDA(cudaMemcpy(J->src.data(), src, m * 4, cudaMemcpyDeviceToHost));
                PGB_CUDA(cudaMemcpy(J->dst.data(), dst, m * 4, cudaMemcpyDeviceToHost));
            }
        }
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) fail(PGB_E_STATE, "server is shutting down");
        J->id = S->next_id++;
        J->submitted = Clock::now();
        S->jobs[J->id] = J;
        S->queued.push_back(J);
        S->cv_queue.notify_all();
        *job_id = J->id;
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
        J->cancel = true;
        auto q = std::find(S->queued.begin(), S->queued.end(), J);
        if (q != S->queued.end()) {
            S->queued.erase(q);
            J->state = PGB_JOB_CANCELLED;
            J->err = PGB_E_CANCELLED;
            J->finished = Clock::now();
            J->src.clear();
            J->dst.clear();
            ++S->n_cancelled;
            S->cv_done.notify_all();
        }
        // a job already on the device runs to the end; its result is dropped
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
        }
        S->queued.clear();
        S->cv_queue.notify_all();
        S->cv_ready.notify_all();
        S->cv_done.notify_all();
    }
    for (auto& t : S->threads) t.join();
    for (auto& J : S->ready) J->release_device();
    S->ready.clear();
    S->jobs.clear();
    for (cudaStream_t st : S->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    delete S;
    live_handles_add(-1);
}

}  // extern "C"
