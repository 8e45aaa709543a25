// Serving engine: continuous admission of component-matrix jobs whose event
// batches arrive over time.
//
// The paper's method is one pass over a time-ordered stream (Section 3.5), so
// a job's state -- its component matrix -- can stay on the device while its
// event batches arrive.  This engine serves many such jobs at once:
//   * tn_server_open registers a job (n nodes, a bound on its batch size, the
//     host buffers of its results) and queues it for admission;
//   * tn_server_push hands the job a batch of host events; batches wait in the
//     job until it is admitted and are applied in push order;
//   * worker threads admit queued jobs in open order whenever a slot is free
//     and the job's device memory fits the budget.  An admitted job owns an
//     online state (tn_online_*: S <- I, then each batch; a timestamp group
//     split by a batch boundary is held back until it is complete) on a
//     stream of its own.  A worker copies a pending batch in and pushes it to
//     the job's state; one worker at a time serves a given job, so its batches
//     keep their order while the other workers serve other jobs;
//   * after the batch marked last, the out-sizes are computed and copied back
//     on the job's stream; a finished job releases its memory and reports its
//     timings through poll().
// Jobs on different streams overlap on the device.  tn_server_submit is
// open + one push per batch.
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
#include <unordered_map>
#include <vector>

#include "tn_internal.cuh"

namespace {

constexpr uint32_t kDefaultWorkers = 16;
constexpr uint64_t kBytesPerBatchEvent = 160;  // copy in 16, held-back group 16, schedule ~128

uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct ServeBatch {
    const uint32_t *u = nullptr, *v = nullptr;
    const int64_t *t = nullptr;
    uint64_t m = 0;
    bool last = false;
};

// The device resources of a resident job, reused by the next job that takes
// the slot (creating and destroying streams, events and buffers per job would
// serialise the workers in the driver): a stream for copies and scheduling, a
// stream for matrix updates, sizes and the copy back, the job's completion
// event, copy-in buffers, result buffers and the pinned staging of the results.
struct ServeSlot {
    cudaStream_t st = nullptr, ast = nullptr;
    cudaEvent_t done = nullptr;
    uint32_t *du = nullptr, *dv = nullptr, *d_out = nullptr, *d_am = nullptr;
    int64_t *dt = nullptr;
    uint32_t *h_pin = nullptr;
    uint64_t cap_events = 0, cap_nodes = 0, cap_pin = 0;
};

struct ServeJob {
    uint64_t id = 0;
    uint32_t n = 0;
    uint64_t max_batch = 0;
    uint32_t *h_out = nullptr, *h_argmax = nullptr;
    uint64_t bytes = 0;  // device bytes charged to the budget
    // guarded by the server's mutex
    std::deque<ServeBatch> batches;  // pushed, not yet applied
    bool closed = false;             // the last batch has been pushed
    bool busy = false;               // a worker is serving one of its batches
    bool finishing = false;          // results enqueued (or the job failed): retire when done
    uint64_t events = 0;
    // device state, used by one worker at a time: copies in and scheduling on
    // slot->st, matrix updates, sizes and the copy back on slot->ast
    ServeSlot *slot = nullptr;
    tn_online *on = nullptr;
    tn_status status = TN_OK;
    uint64_t t_open = 0, t_admit = 0, t_last_push = 0, t_enqueued = 0, t_done = 0;
};

}  // namespace

struct tn_server {
    int device = 0;
    tn_server_options opt{};
    uint64_t budget = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::unordered_map<uint64_t, ServeJob *> open;  // opened, not yet retired
    std::deque<ServeJob *> queue;                   // waiting for admission, in open order
    std::vector<ServeJob *> active;                 // admitted
    std::deque<tn_job_record> finished;
    std::condition_variable finished_cv;
    uint64_t in_use = 0;
    uint64_t admitted = 0, completed = 0, peak_active = 0, peak_bytes = 0;
    std::atomic<uint64_t> batches{0}, admit_ns{0}, copy_ns{0}, schedule_ns{0}, result_ns{0}, retire_ns{0};
    uint64_t starting = 0;  // admissions in progress
    bool stop = false;
    std::vector<std::thread> workers;
    std::vector<ServeSlot *> slots;  // free slots of finished jobs
};

namespace {

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
constexpr uint32_t kServeWindow = 576;
constexpr uint32_t kServeRowBytes = 144 * 1024;

uint32_t serve_slab_words(uint32_t n)
{
    const uint64_t ld = tn_row_words(n);
    uint64_t sw = ld / 16;
    if (sw > 16) sw = 16;
    sw &= ~1ull;
    return sw < 2 ? 2u : (uint32_t)sw;
}

ServeSlot *take_slot(tn_server *s)
{
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (!s->slots.empty()) {
            ServeSlot *sl = s->slots.back();
            s->slots.pop_back();
            return sl;
        }
    }
    ServeSlot *sl = new (std::nothrow) ServeSlot();
    if (!sl) return nullptr;
    // scheduling (short kernels the worker waits for) before matrix updates
    // (long-running CTAs): highest priority for st, lowest for ast
    int least = 0, greatest = 0;
    cudaError_t err = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (err == cudaSuccess) err = cudaStreamCreateWithPriority(&sl->st, cudaStreamNonBlocking, greatest);
    if (err == cudaSuccess) err = cudaStreamCreateWithPriority(&sl->ast, cudaStreamNonBlocking, least);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&sl->done, cudaEventDisableTiming);
    if (err != cudaSuccess) {
        tn_internal_set_cuda_error(err);
        if (sl->done) cudaEventDestroy(sl->done);
        if (sl->ast) cudaStreamDestroy(sl->ast);
        if (sl->st) cudaStreamDestroy(sl->st);
        delete sl;
        return nullptr;
    }
    return sl;
}

void free_slot(ServeSlot *sl)
{
    if (sl->du) cudaFreeAsync(sl->du, sl->st);
    if (sl->dv) cudaFreeAsync(sl->dv, sl->st);
    if (sl->dt) cudaFreeAsync(sl->dt, sl->st);
    if (sl->d_out) cudaFreeAsync(sl->d_out, sl->ast);
    if (sl->d_am) cudaFreeAsync(sl->d_am, sl->ast);
    if (sl->st) cudaStreamSynchronize(sl->st);
    if (sl->ast) cudaStreamSynchronize(sl->ast);
    if (sl->h_pin) cudaFreeHost(sl->h_pin);
    if (sl->done) cudaEventDestroy(sl->done);
    if (sl->ast) cudaStreamDestroy(sl->ast);
    if (sl->st) cudaStreamDestroy(sl->st);
    delete sl;
}

// Buffers of a slot large enough for this job; they only grow.  Device buffers
// come from the stream-ordered pool on the slot's own streams (a plain free
// would synchronise the device); the pinned staging is rounded up to a power
// of two of at least 64 Ki entries, so it rarely grows.
tn_status fit_slot(ServeSlot *sl, uint64_t max_batch, uint32_t n)
{
    const uint64_t mb = max_batch ? max_batch : 1;
    if (sl->cap_events < mb) {
        if (sl->du) cudaFreeAsync(sl->du, sl->st);
        if (sl->dv) cudaFreeAsync(sl->dv, sl->st);
        if (sl->dt) cudaFreeAsync(sl->dt, sl->st);
        sl->du = sl->dv = nullptr;
        sl->dt = nullptr;
        sl->cap_events = 0;
        SERVE_TRY(cudaMallocAsync((void **)&sl->du, mb * 4, sl->st));
        SERVE_TRY(cudaMallocAsync((void **)&sl->dv, mb * 4, sl->st));
        SERVE_TRY(cudaMallocAsync((void **)&sl->dt, mb * 8, sl->st));
        sl->cap_events = mb;
    }
    if (sl->cap_nodes < n) {
        if (sl->d_out) cudaFreeAsync(sl->d_out, sl->ast);
        sl->d_out = nullptr;
        sl->cap_nodes = 0;
        if (!sl->d_am) SERVE_TRY(cudaMallocAsync((void **)&sl->d_am, 4, sl->ast));
        SERVE_TRY(cudaMallocAsync((void **)&sl->d_out, (uint64_t)n * 4, sl->ast));
        sl->cap_nodes = n;
    }
    if (sl->cap_pin < (uint64_t)n + 2) {  // sizes, argmax, status
        uint64_t c = 1ull << 16;
        while (c < (uint64_t)n + 2) c *= 2;
        if (sl->h_pin) cudaFreeHost(sl->h_pin);
        sl->h_pin = nullptr;
        sl->cap_pin = 0;
        SERVE_TRY(cudaHostAlloc((void **)&sl->h_pin, c * 4, cudaHostAllocDefault));
        sl->cap_pin = c;
    }
    return TN_OK;
}

// Slot (streams, buffers) and online state (two-stream mode) of an admitted job.
tn_status start_job(tn_server *s, ServeJob *j)
{
    j->slot = take_slot(s);
    if (!j->slot) return TN_ECUDA;
    ServeSlot *sl = j->slot;
    tn_status rc = fit_slot(sl, j->max_batch, j->n);
    if (rc != TN_OK) return rc;
    tn_plan_options opt;
    memset(&opt, 0, sizeof(opt));
    opt.window_events = s->opt.window_events;
    opt.slab_words = s->opt.slab_words ? s->opt.slab_words : serve_slab_words(j->n);
    if (!opt.window_events) {
        // Room on every SM for the scheduler's CTAs beside a running update
        // CTA, so that a batch's schedule does not wait for an SM to free up:
        // windows of kServeWindow events (a 36 KB scheduling arena) and a row
        // buffer of kServeRowBytes (the 2 x kServeWindow rows such a window can
        // touch, at 16-word slabs)
        opt.window_events = kServeWindow;
        opt.smem_rows = kServeRowBytes / (8u * opt.slab_words);
    }
    rc = tn_online_create(j->n, &opt, sl->ast, &j->on);
    if (rc != TN_OK) return rc;
    rc = tn::online_use_apply_stream(j->on, sl->ast);
    if (rc != TN_OK) return rc;
    // the state's and the slot's buffers are ready for both streams
    SERVE_TRY(tn_internal_stream_wait(sl->ast));
    SERVE_TRY(tn_internal_stream_wait(sl->st));
    return TN_OK;
}

// One batch of an admitted job: copy in, push to the online state, and after
// the last batch the out-sizes and their copy to the caller.
tn_status serve_batch(tn_server *s, ServeJob *j, const ServeBatch &b)
{
    ServeSlot *sl = j->slot;
    const uint64_t t0 = now_ns();
    if (b.m) {
        SERVE_TRY(cudaMemcpyAsync(sl->du, b.u, b.m * 4, cudaMemcpyHostToDevice, sl->st));
        SERVE_TRY(cudaMemcpyAsync(sl->dv, b.v, b.m * 4, cudaMemcpyHostToDevice, sl->st));
        SERVE_TRY(cudaMemcpyAsync(sl->dt, b.t, b.m * 8, cudaMemcpyHostToDevice, sl->st));
    }
    const uint64_t t1 = now_ns();
    tn_status rc = tn_online_push(j->on, sl->du, sl->dv, sl->dt, b.m, b.last ? TN_GROUP_END : 0u, sl->st);
    const uint64_t t2 = now_ns();
    s->copy_ns += t1 - t0;
    s->schedule_ns += t2 - t1;
    s->batches++;
    if (rc != TN_OK || !b.last) return rc;
    tn_online_state state;
    rc = tn_online_get_state(j->on, &state);
    if (rc != TN_OK) return rc;
    rc = tn_out_sizes(state.S, j->n, j->n, sl->d_out, nullptr, sl->d_am, sl->ast);
    if (rc != TN_OK) return rc;
    // into pinned staging: the copy runs behind the updates without blocking
    // this worker; the retiring worker hands the results to the caller
    SERVE_TRY(cudaMemcpyAsync(sl->h_pin, sl->d_out, (uint64_t)j->n * 4, cudaMemcpyDeviceToHost, sl->ast));
    SERVE_TRY(cudaMemcpyAsync(sl->h_pin + j->n, sl->d_am, 4, cudaMemcpyDeviceToHost, sl->ast));
    SERVE_TRY(cudaMemcpyAsync(sl->h_pin + j->n + 1, tn::online_status_word(j->on), 4, cudaMemcpyDeviceToHost,
                              sl->ast));
    s->result_ns += now_ns() - t2;
    return TN_OK;
}

// Frees the job's online state (stream-ordered, behind its work) and returns
// its slot to the pool.
void release_job(tn_server *s, ServeJob *j)
{
    if (j->on) tn_online_destroy(j->on, j->slot->st);
    j->on = nullptr;
    if (j->slot) {
        std::lock_guard<std::mutex> lock(s->mu);
        s->slots.push_back(j->slot);
    }
    j->slot = nullptr;
}

void finish_job(tn_server *s, ServeJob *j)
{
    // a device error of an applied batch: the online state's status word, copied
    // behind the updates with the results (no synchronisation here)
    if (j->status == TN_OK && j->slot) j->status = (tn_status)(int32_t)j->slot->h_pin[j->n + 1];
    if (j->status == TN_OK && j->slot) {  // the job's results reached the staging buffer
        memcpy(j->h_out, j->slot->h_pin, (size_t)j->n * 4);
        if (j->h_argmax) *j->h_argmax = j->slot->h_pin[j->n];
    }
    j->t_done = now_ns();
    tn_job_record r;
    memset(&r, 0, sizeof(r));
    r.job_id = j->id;
    r.status = j->status;
    r.n = j->n;
    r.events = j->events;
    r.t_submit_ns = j->t_open;
    r.t_admit_ns = j->t_admit;
    r.t_done_ns = j->t_done;
    r.t_last_push_ns = j->t_last_push;
    r.t_enqueued_ns = j->t_enqueued;
    release_job(s, j);
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->in_use -= j->bytes;
        s->completed++;
        s->finished.push_back(r);
    }
    s->finished_cv.notify_all();
    delete j;
}

// Admits the head of the queue if a slot and the memory are free.
bool admit_one(tn_server *s)
{
    ServeJob *j = nullptr;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        const uint64_t resident = s->active.size() + s->starting;
        if (s->queue.empty() || resident >= s->opt.max_active) return false;
        ServeJob *head = s->queue.front();
        // bytes stay charged until a retired job's memory is released (a job
        // larger than the budget was refused at open, so with nothing charged
        // the head always fits)
        if (s->in_use + head->bytes > s->budget) return false;
        s->queue.pop_front();
        s->in_use += head->bytes;
        s->admitted++;
        s->starting++;
        j = head;
    }
    j->t_admit = now_ns();
    const tn_status rc = start_job(s, j);
    s->admit_ns += now_ns() - j->t_admit;
    std::lock_guard<std::mutex> lock(s->mu);
    if (rc != TN_OK) j->status = rc;
    s->starting--;
    s->active.push_back(j);
    if (s->active.size() > s->peak_active) s->peak_active = s->active.size();
    if (s->in_use > s->peak_bytes) s->peak_bytes = s->in_use;
    return true;
}

// Serves the next pending batch of some admitted job that no other worker is
// serving.  A failed job drops its batches and finishes at its last one.
bool serve_one(tn_server *s)
{
    ServeJob *j = nullptr;
    ServeBatch b;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        for (ServeJob *c : s->active) {
            if (c->busy || c->finishing || c->batches.empty()) continue;
            j = c;
            b = c->batches.front();
            c->batches.pop_front();
            c->busy = true;
            break;
        }
    }
    if (!j) return false;
    if (j->status == TN_OK) j->status = serve_batch(s, j, b);
    if (b.last && j->slot) cudaEventRecord(j->slot->done, j->slot->ast);
    std::lock_guard<std::mutex> lock(s->mu);
    j->busy = false;
    if (b.last) {
        j->finishing = true;
        j->t_enqueued = now_ns();
    }
    return true;
}

// Retires the admitted jobs whose results have reached the host.
bool retire_done(tn_server *s)
{
    std::vector<ServeJob *> done;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        for (size_t i = 0; i < s->active.size();) {
            ServeJob *j = s->active[i];
            const bool ready = j->finishing && !j->busy &&
                               (!j->slot || cudaEventQuery(j->slot->done) != cudaErrorNotReady);
            if (ready) {
                done.push_back(j);
                s->open.erase(j->id);
                s->active[i] = s->active.back();
                s->active.pop_back();
            } else {
                ++i;
            }
        }
    }
    const uint64_t t0 = now_ns();
    for (ServeJob *j : done) finish_job(s, j);
    if (!done.empty()) s->retire_ns += now_ns() - t0;
    return !done.empty();
}

void worker_loop(tn_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        bool progressed = false;
        while (admit_one(s)) progressed = true;
        while (serve_one(s)) progressed = true;
        progressed = retire_done(s) || progressed;
        std::unique_lock<std::mutex> lock(s->mu);
        if (s->stop && s->starting == 0) {
            // after tn_server_destroy: run every job whose last batch was pushed
            bool waiting = false;
            for (ServeJob *q : s->queue) waiting = waiting || q->closed;
            for (ServeJob *a : s->active) waiting = waiting || a->closed;
            if (!waiting) return;
        }
        if (!progressed) {
            if (s->active.empty()) {
                s->cv.wait_for(lock, std::chrono::milliseconds(2));
            } else {
                lock.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            }
        }
    }
}

}  // namespace

extern "C" uint64_t tn_server_job_bytes(uint32_t n, uint64_t max_batch_events)
{
    const uint64_t rows = ((uint64_t)n + 1023) / 1024 * 1024;
    return rows * tn_row_words(n) * 8 + (uint64_t)n * 4 + 256 + max_batch_events * kBytesPerBatchEvent;
}

extern "C" tn_status tn_server_create(const tn_server_options *opt, tn_server **out)
{
    if (!out) return TN_EINVAL;
    *out = nullptr;
    if (opt && (opt->reserved[0] || opt->reserved[1])) return TN_EINVAL;
    tn_server *s = new (std::nothrow) tn_server();
    if (!s) return TN_ENOMEM;
    if (opt) s->opt = *opt;
    if (s->opt.max_active == 0) s->opt.max_active = 16;
    if (s->opt.workers == 0) s->opt.workers = kDefaultWorkers;
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
    // several workers, so that copying in and scheduling one job's batch (host
    // synchronisations on its own stream) does not hold up the others
    for (uint32_t w = 0; w < s->opt.workers; ++w) s->workers.emplace_back(worker_loop, s);
    *out = s;
    return TN_OK;
}

extern "C" tn_status tn_server_open(tn_server *s, uint64_t job_id, uint32_t n, uint64_t max_batch_events,
                                    uint32_t *out_sizes, uint32_t *argmax)
{
    if (!s || n == 0 || n >= (1u << 30) || !out_sizes || max_batch_events >= (1ull << 30)) return TN_EINVAL;
    ServeJob *j = new (std::nothrow) ServeJob();
    if (!j) return TN_ENOMEM;
    j->id = job_id;
    j->n = n;
    j->max_batch = max_batch_events;
    j->h_out = out_sizes;
    j->h_argmax = argmax;
    j->bytes = tn_server_job_bytes(n, max_batch_events);
    j->t_open = now_ns();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        tn_status rc = TN_OK;
        if (j->bytes > s->budget) rc = TN_ENOMEM;  // could never be admitted
        else if (s->stop || s->open.count(job_id)) rc = TN_EINVAL;
        if (rc != TN_OK) {
            delete j;
            return rc;
        }
        s->open[job_id] = j;
        s->queue.push_back(j);
    }
    s->cv.notify_all();
    return TN_OK;
}

extern "C" tn_status tn_server_push(tn_server *s, uint64_t job_id, const uint32_t *u, const uint32_t *v,
                                    const int64_t *t, uint64_t m, uint32_t flags)
{
    if (!s || (flags & ~TN_LAST_BATCH) || (m > 0 && (!u || !v || !t))) return TN_EINVAL;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        auto it = s->open.find(job_id);
        if (it == s->open.end()) return TN_EINVAL;
        ServeJob *j = it->second;
        if (j->closed || m > j->max_batch) return TN_EINVAL;
        ServeBatch b;
        b.u = u;
        b.v = v;
        b.t = t;
        b.m = m;
        b.last = (flags & TN_LAST_BATCH) != 0;
        try {
            j->batches.push_back(b);
        } catch (...) {
            return TN_ENOMEM;
        }
        j->events += m;
        if (b.last) {
            j->closed = true;
            j->t_last_push = now_ns();
        }
    }
    s->cv.notify_all();
    return TN_OK;
}

extern "C" tn_status tn_server_submit(tn_server *s, uint64_t job_id, uint32_t n, const uint32_t *u,
                                      const uint32_t *v, const int64_t *t, const uint64_t *batch_offsets,
                                      uint32_t nbatches, uint32_t *out_sizes, uint32_t *argmax)
{
    if (!s || n == 0 || n >= (1u << 30) || !batch_offsets || nbatches == 0 || !out_sizes) return TN_EINVAL;
    const uint64_t m = batch_offsets[nbatches];
    if (batch_offsets[0] != 0 || (m > 0 && (!u || !v || !t))) return TN_EINVAL;
    uint64_t max_batch = 0;
    for (uint32_t b = 0; b < nbatches; ++b) {
        if (batch_offsets[b + 1] < batch_offsets[b]) return TN_EINVAL;
        const uint64_t mb = batch_offsets[b + 1] - batch_offsets[b];
        if (mb >= (1ull << 30)) return TN_EINVAL;
        if (mb > max_batch) max_batch = mb;
    }
    tn_status rc = tn_server_open(s, job_id, n, max_batch, out_sizes, argmax);
    if (rc != TN_OK) return rc;
    for (uint32_t b = 0; b < nbatches && rc == TN_OK; ++b) {
        const uint64_t e0 = batch_offsets[b];
        rc = tn_server_push(s, job_id, u + e0, v + e0, t + e0, batch_offsets[b + 1] - e0,
                            b + 1 == nbatches ? TN_LAST_BATCH : 0u);
    }
    if (rc != TN_OK) {
        // the job ends with this error: its pushed batches are dropped unread
        // (the caller is told to release its buffers) and its record reports rc
        std::lock_guard<std::mutex> lock(s->mu);
        auto it = s->open.find(job_id);
        if (it != s->open.end()) {
            ServeJob *j = it->second;
            j->status = rc;
            j->batches.clear();
            j->closed = true;
            ServeBatch end;
            end.last = true;
            j->batches.push_back(end);
        }
    }
    return rc;
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
    out->batches = s->batches;
    out->admit_ns = s->admit_ns;
    out->copy_ns = s->copy_ns;
    out->schedule_ns = s->schedule_ns;
    out->result_ns = s->result_ns;
    out->retire_ns = s->retire_ns;
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
    // jobs that never received their last batch (never admitted, or admitted
    // and waiting): their matrices are released without results
    for (auto &kv : s->open) {
        ServeJob *j = kv.second;
        release_job(s, j);
        delete j;
    }
    for (ServeSlot *sl : s->slots) free_slot(sl);
    delete s;
    return TN_OK;
}
