// Serving engine: continuous admission of component-matrix jobs.
//
// The paper's method is a streaming algorithm (Section 3.5): new events are
// applied to the stored component matrix with the same rule, so a job's state
// (its matrix S) can live on the device across incremental event batches.
// This engine serves many such jobs at once:
//   * submit() queues a job (n nodes, its events split into batches of
//     increasing time) together with the host buffer its out-sizes go to;
//   * a worker thread admits queued jobs in arrival order whenever a slot is
//     free and the job's device memory fits the budget, so jobs that arrive
//     while others run join the device as soon as memory frees up;
//   * an admitted job gets its own stream: its events are copied in, every
//     batch is scheduled (tn_plan_create), and the batches are applied in
//     order to the same S with the t_last order gate, followed by the
//     out-sizes and the copy back.  Jobs on different streams overlap on the
//     device.  A batch boundary inside a timestamp group is moved to the end
//     of the group at submit, so each group is applied whole;
//   * finished jobs release their memory and report timings through poll().
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "tn_internal.cuh"

namespace {

constexpr int kServeWorkers = 4;

uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct ServeJob {
    uint64_t id = 0;
    uint32_t n = 0;
    const uint32_t *hu = nullptr, *hv = nullptr;
    const int64_t *ht = nullptr;
    std::vector<uint64_t> offs;  // batch b = events [offs[b], offs[b+1])
    uint32_t *h_out = nullptr, *h_argmax = nullptr;
    uint64_t bytes = 0;  // device bytes charged to the budget
    // device state
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    uint64_t *S = nullptr;
    int64_t *t_last = nullptr;
    uint32_t *d_out = nullptr, *d_am = nullptr;
    std::vector<tn_plan *> plans;
    tn_status status = TN_OK;
    uint64_t t_submit = 0, t_admit = 0, t_done = 0;
};

}  // namespace

struct tn_server {
    int device = 0;
    tn_server_options opt{};
    uint64_t budget = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<ServeJob *> queue;
    std::vector<ServeJob *> active;
    std::deque<tn_job_record> finished;
    std::condition_variable finished_cv;
    uint64_t in_use = 0;
    uint64_t admitted = 0, completed = 0, peak_active = 0, peak_bytes = 0;
    uint64_t starting = 0;  // jobs admitted whose start is in progress
    bool stop = false;
    std::vector<std::thread> workers;
};

namespace {

uint64_t job_bytes(uint32_t n, uint64_t m, uint64_t max_batch)
{
    // matrix + sizes + t_last, the largest batch's events while its plan is
    // built, and the schedules (about 16 bytes per event, 64 while building)
    return (uint64_t)n * tn_row_words(n) * 8 + (uint64_t)n * 4 + 64 + max_batch * 16 + m * 16 + max_batch * 64;
}

void release_job(ServeJob *j)
{
    for (tn_plan *p : j->plans)
        if (p) tn_plan_destroy(p, j->st);
    if (j->S) cudaFreeAsync(j->S, j->st);
    if (j->t_last) cudaFreeAsync(j->t_last, j->st);
    if (j->d_out) cudaFreeAsync(j->d_out, j->st);
    if (j->d_am) cudaFreeAsync(j->d_am, j->st);
    if (j->st) cudaStreamSynchronize(j->st);
    if (j->done) cudaEventDestroy(j->done);
    if (j->st) cudaStreamDestroy(j->st);
}

#define SERVE_TRY(expr)                           \
    do {                                          \
        cudaError_t e_ = (expr);                  \
        if (e_ != cudaSuccess) {                  \
            tn_internal_set_cuda_error(e_);       \
            return e_ == cudaErrorMemoryAllocation ? TN_ENOMEM : TN_ECUDA; \
        }                                         \
    } while (0)

// Slab width of a job when the server options leave it open: a small matrix
// still gets at least 16 CTAs (every CTA streams all of the job's events, so
// narrower slabs shorten the job), large ones keep 16-word slabs.
uint32_t serve_slab_words(uint32_t n)
{
    const uint64_t ld = tn_row_words(n);
    uint64_t sw = ld / 16;
    if (sw > 16) sw = 16;
    sw &= ~1ull;
    return sw < 2 ? 2u : (uint32_t)sw;
}

// Copies the job in, schedules every batch and enqueues the whole job on its
// stream.  Runs on the worker thread.
tn_status start_job(tn_server *s, ServeJob *j)
{
    SERVE_TRY(cudaStreamCreateWithFlags(&j->st, cudaStreamNonBlocking));
    SERVE_TRY(cudaEventCreateWithFlags(&j->done, cudaEventDisableTiming));
    const uint64_t ld = tn_row_words(j->n);
    const uint32_t nb = (uint32_t)j->offs.size() - 1;
    SERVE_TRY(cudaMallocAsync((void **)&j->S, (uint64_t)j->n * ld * 8, j->st));
    SERVE_TRY(cudaMallocAsync((void **)&j->t_last, sizeof(int64_t), j->st));
    SERVE_TRY(cudaMallocAsync((void **)&j->d_out, (uint64_t)j->n * 4, j->st));
    SERVE_TRY(cudaMallocAsync((void **)&j->d_am, 4, j->st));
    // schedules of all batches (they depend on the events only)
    uint64_t max_batch = 0;
    for (uint32_t b = 0; b < nb; ++b)
        if (j->offs[b + 1] - j->offs[b] > max_batch) max_batch = j->offs[b + 1] - j->offs[b];
    uint32_t *du = nullptr, *dv = nullptr;
    int64_t *dt = nullptr;
    if (max_batch) {
        SERVE_TRY(cudaMallocAsync((void **)&du, max_batch * 4, j->st));
        SERVE_TRY(cudaMallocAsync((void **)&dv, max_batch * 4, j->st));
        SERVE_TRY(cudaMallocAsync((void **)&dt, max_batch * 8, j->st));
    }
    tn_plan_options opt;
    memset(&opt, 0, sizeof(opt));
    opt.window_events = s->opt.window_events;
    opt.slab_words = s->opt.slab_words ? s->opt.slab_words : serve_slab_words(j->n);
    tn_status rc = TN_OK;
    for (uint32_t b = 0; b < nb && rc == TN_OK; ++b) {
        const uint64_t e0 = j->offs[b], mb = j->offs[b + 1] - e0;
        if (mb == 0) {
            j->plans.push_back(nullptr);
            continue;
        }
        cudaError_t err = cudaMemcpyAsync(du, j->hu + e0, mb * 4, cudaMemcpyHostToDevice, j->st);
        if (err == cudaSuccess) err = cudaMemcpyAsync(dv, j->hv + e0, mb * 4, cudaMemcpyHostToDevice, j->st);
        if (err == cudaSuccess) err = cudaMemcpyAsync(dt, j->ht + e0, mb * 8, cudaMemcpyHostToDevice, j->st);
        if (err != cudaSuccess) {
            tn_internal_set_cuda_error(err);
            rc = TN_ECUDA;
            break;
        }
        tn_plan *p = nullptr;
        rc = tn_plan_create(du, dv, dt, mb, j->n, nullptr, &opt, j->st, &p);
        j->plans.push_back(p);
    }
    if (du) cudaFreeAsync(du, j->st);
    if (dv) cudaFreeAsync(dv, j->st);
    if (dt) cudaFreeAsync(dt, j->st);
    if (rc != TN_OK) return rc;
    // S <- I, then the batches in order; t_last orders them on the device
    const int64_t lowest = INT64_MIN;
    SERVE_TRY(cudaMemcpyAsync(j->t_last, &lowest, sizeof(lowest), cudaMemcpyHostToDevice, j->st));
    bool first = true;
    for (tn_plan *p : j->plans) {
        if (!p) continue;
        rc = tn_plan_apply(p, j->S, j->n, nullptr, j->t_last, first ? TN_INIT_IDENTITY : 0u, j->st);
        if (rc != TN_OK) return rc;
        first = false;
    }
    if (first) {  // no events at all: the identity
        rc = tn_init_matrix(j->S, j->n, j->n, nullptr, j->st);
        if (rc != TN_OK) return rc;
    }
    rc = tn_out_sizes(j->S, j->n, j->n, j->d_out, nullptr, j->d_am, j->st);
    if (rc != TN_OK) return rc;
    SERVE_TRY(cudaMemcpyAsync(j->h_out, j->d_out, (uint64_t)j->n * 4, cudaMemcpyDeviceToHost, j->st));
    if (j->h_argmax) SERVE_TRY(cudaMemcpyAsync(j->h_argmax, j->d_am, 4, cudaMemcpyDeviceToHost, j->st));
    SERVE_TRY(cudaEventRecord(j->done, j->st));
    return TN_OK;
}

void finish_job(tn_server *s, ServeJob *j)
{
    j->t_done = now_ns();
    // errors recorded by the kernels (batch order) live in the plans
    for (tn_plan *p : j->plans) {
        if (!p) continue;
        const tn_status ps = tn_plan_status(p, j->st);
        if (j->status == TN_OK && ps != TN_OK) j->status = ps;
    }
    tn_job_record r;
    memset(&r, 0, sizeof(r));
    r.job_id = j->id;
    r.status = j->status;
    r.n = j->n;
    r.events = j->offs.back();
    r.t_submit_ns = j->t_submit;
    r.t_admit_ns = j->t_admit;
    r.t_done_ns = j->t_done;
    release_job(j);
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->in_use -= j->bytes;
        s->completed++;
        s->finished.push_back(r);
    }
    s->finished_cv.notify_all();
    delete j;
}

void worker_loop(tn_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        bool progressed = false;
        // admit in arrival order while a slot and the memory are free
        for (;;) {
            ServeJob *j = nullptr;
            {
                std::lock_guard<std::mutex> lock(s->mu);
                const uint64_t resident = s->active.size() + s->starting;
                if (s->queue.empty() || resident >= s->opt.max_active) break;
                ServeJob *head = s->queue.front();
                if (s->in_use + head->bytes > s->budget && resident > 0) break;
                s->queue.pop_front();
                s->in_use += head->bytes;
                s->admitted++;
                s->starting++;
                j = head;
            }
            j->t_admit = now_ns();
            j->status = start_job(s, j);
            std::lock_guard<std::mutex> lock(s->mu);
            s->starting--;
            s->active.push_back(j);
            if (s->active.size() > s->peak_active) s->peak_active = s->active.size();
            if (s->in_use > s->peak_bytes) s->peak_bytes = s->in_use;
            progressed = true;
        }
        // retire finished jobs
        std::vector<ServeJob *> done;
        {
            std::lock_guard<std::mutex> lock(s->mu);
            for (size_t i = 0; i < s->active.size();) {
                ServeJob *j = s->active[i];
                const bool ready = j->status != TN_OK || cudaEventQuery(j->done) != cudaErrorNotReady;
                if (ready) {
                    done.push_back(j);
                    s->active[i] = s->active.back();
                    s->active.pop_back();
                } else {
                    ++i;
                }
            }
        }
        for (ServeJob *j : done) finish_job(s, j);
        progressed = progressed || !done.empty();
        {
            std::unique_lock<std::mutex> lock(s->mu);
            if (s->stop && s->queue.empty() && s->active.empty() && s->starting == 0) return;
            if (!progressed) {
                if (s->active.empty()) {
                    s->cv.wait_for(lock, std::chrono::milliseconds(5));
                } else {
                    lock.unlock();
                    std::this_thread::sleep_for(std::chrono::microseconds(20));
                }
            }
        }
    }
}

}  // namespace

extern "C" tn_status tn_server_create(const tn_server_options *opt, tn_server **out)
{
    if (!out) return TN_EINVAL;
    *out = nullptr;
    tn_server *s = new (std::nothrow) tn_server();
    if (!s) return TN_ENOMEM;
    if (opt) s->opt = *opt;
    if (s->opt.max_active == 0) s->opt.max_active = 16;
    cudaError_t err = cudaGetDevice(&s->device);
    size_t free_b = 0, total_b = 0;
    if (err == cudaSuccess) err = cudaMemGetInfo(&free_b, &total_b);
    if (err != cudaSuccess) {
        tn_internal_set_cuda_error(err);
        delete s;
        return TN_ECUDA;
    }
    tn_internal_keep_pool();
    s->budget = s->opt.memory_budget ? s->opt.memory_budget : (uint64_t)(free_b * 0.6);
    // several workers, so that copying in and scheduling one job (host
    // synchronisations on its own stream) does not hold up the admission of
    // the next ones
    for (int w = 0; w < kServeWorkers; ++w) s->workers.emplace_back(worker_loop, s);
    *out = s;
    return TN_OK;
}

extern "C" tn_status tn_server_submit(tn_server *s, uint64_t job_id, uint32_t n, const uint32_t *u,
                                      const uint32_t *v, const int64_t *t, const uint64_t *batch_offsets,
                                      uint32_t nbatches, uint32_t *out_sizes, uint32_t *argmax)
{
    if (!s || n == 0 || n >= (1u << 30) || !batch_offsets || nbatches == 0 || !out_sizes) return TN_EINVAL;
    const uint64_t m = batch_offsets[nbatches];
    if (batch_offsets[0] != 0 || (m > 0 && (!u || !v || !t))) return TN_EINVAL;
    for (uint32_t b = 0; b < nbatches; ++b)
        if (batch_offsets[b + 1] < batch_offsets[b]) return TN_EINVAL;
    std::vector<uint64_t> offs;
    try {
        offs.assign(batch_offsets, batch_offsets + nbatches + 1);
    } catch (...) {
        return TN_ENOMEM;
    }
    // A timestamp group is one snapshot (Section 2.1), so it must be applied
    // whole: a batch boundary inside a group moves to the group's end, and the
    // group is applied with the next batch (as the online state holds it back).
    for (uint32_t b = 1; b < nbatches; ++b) {
        uint64_t x = offs[b] > offs[b - 1] ? offs[b] : offs[b - 1];
        while (x > 0 && x < m && t[x] == t[x - 1]) ++x;
        offs[b] = x;
    }
    uint64_t max_batch = 0;
    for (uint32_t b = 0; b < nbatches; ++b) {
        const uint64_t mb = offs[b + 1] - offs[b];
        if (mb >= (1ull << 30)) return TN_EINVAL;
        if (mb > max_batch) max_batch = mb;
    }
    ServeJob *j = new (std::nothrow) ServeJob();
    if (!j) return TN_ENOMEM;
    j->id = job_id;
    j->n = n;
    j->hu = u;
    j->hv = v;
    j->ht = t;
    j->offs.swap(offs);
    j->h_out = out_sizes;
    j->h_argmax = argmax;
    j->bytes = job_bytes(n, m, max_batch);
    j->t_submit = now_ns();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (j->bytes > s->budget) {
            delete j;
            return TN_ENOMEM;  // could never be admitted
        }
        if (s->stop) {
            delete j;
            return TN_EINVAL;
        }
        s->queue.push_back(j);
    }
    s->cv.notify_all();
    return TN_OK;
}

extern "C" tn_status tn_server_poll(tn_server *s, tn_job_record *records, uint32_t capacity, uint32_t *count,
                                    uint32_t wait_ms)
{
    if (!s || !count || (capacity && !records)) return TN_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->finished.empty() && wait_ms)
        s->finished_cv.wait_for(lock, std::chrono::milliseconds(wait_ms), [&] { return !s->finished.empty(); });
    uint32_t c = 0;
    while (c < capacity && !s->finished.empty()) {
        records[c++] = s->finished.front();
        s->finished.pop_front();
    }
    *count = c;
    return TN_OK;
}

extern "C" tn_status tn_server_get_stats(tn_server *s, tn_server_stats *out)
{
    if (!s || !out) return TN_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    memset(out, 0, sizeof(*out));
    out->queued = s->queue.size();
    out->active = s->active.size();
    out->admitted = s->admitted;
    out->completed = s->completed;
    out->bytes_in_use = s->in_use;
    out->budget = s->budget;
    out->peak_active = s->peak_active;
    out->peak_bytes = s->peak_bytes;
    return TN_OK;
}

extern "C" tn_status tn_server_destroy(tn_server *s)
{
    if (!s) return TN_EINVAL;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    for (std::thread &w : s->workers)
        if (w.joinable()) w.join();
    delete s;
    return TN_OK;
}
