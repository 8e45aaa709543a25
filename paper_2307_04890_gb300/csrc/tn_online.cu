// Online streaming state (Section 3.5, advantages and limitations of the matrix
// method): a component matrix that stays on the device while event batches and
// new nodes arrive.
//
//  * Node growth: a new node brings a row and a column of zeros with only its
//    own diagonal bit set.  grow_kernel rewrites a matrix in the padded row layout for
//    more nodes; when the row stride is unchanged it only touches the new rows
//    and the new columns of the old rows.
//  * Timestamp groups split across batches: a group is one snapshot (every
//    event of it reads the rows as they were before the group), so a group may
//    only be applied once all of its events are known.  The online state holds
//    the events of the last timestamp of every pushed batch back ("pending")
//    and applies them together with the next batch (whose first events may
//    continue the same group), or when the caller says the group is complete.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "tn_internal.cuh"

namespace {

// ---------------------------------------------------------------------------
// growth: rows [row0, row1) and words [w0, W_new) of S_new
//   word (i, w) = S_old(i, w) restricted to columns < n_old     (i < n_old)
//               | diagonal bit of row i                         (i >= n_old)
// S_old may equal S_new (same stride): each thread reads and writes only its
// own 16-byte pair.  W_old, W_new and w0 are even (rows are whole 128-byte
// lines), so every pair is 16-byte aligned.
// ---------------------------------------------------------------------------
__global__ void grow_kernel(const uint64_t *S_old, uint64_t W_old, uint32_t n_old, uint64_t *S_new, uint64_t W_new,
                            uint32_t row0, uint32_t row1, uint64_t w0)
{
    const uint64_t pairs_per_row = (W_new - w0) / 2;
    const uint64_t total = (uint64_t)(row1 - row0) * pairs_per_row;
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < total;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t i = row0 + (uint32_t)(p / pairs_per_row);
        const uint64_t w = w0 + 2 * (p % pairs_per_row);
        uint64_t x = 0, y = 0;
        if (i < n_old && w < W_old) {
            const ulonglong2 o = *reinterpret_cast<const ulonglong2 *>(S_old + (uint64_t)i * W_old + w);
            // keep columns < n_old only
            const int64_t keep0 = (int64_t)n_old - (int64_t)(64 * w);
            const int64_t keep1 = keep0 - 64;
            x = keep0 >= 64 ? o.x : keep0 <= 0 ? 0ull : o.x & ((1ull << keep0) - 1ull);
            y = keep1 >= 64 ? o.y : keep1 <= 0 ? 0ull : o.y & ((1ull << keep1) - 1ull);
        }
        if (i >= n_old) {
            if (i / 64 == w) x |= 1ull << (i % 64);
            if (i / 64 == w + 1) y |= 1ull << (i % 64);
        }
        ulonglong2 r;
        r.x = x;
        r.y = y;
        *reinterpret_cast<ulonglong2 *>(S_new + (uint64_t)i * W_new + w) = r;
    }
}

int grow_blocks(uint64_t pairs)
{
    const uint64_t b = (pairs + 255) / 256;
    const uint64_t cap = 152ull * 8;  // grid-stride over 8 CTAs of 256 threads per SM
    return (int)(b < 1 ? 1 : b < cap ? b : cap);
}

tn_status launch_grow(const uint64_t *S_old, uint32_t n_old, uint64_t *S_new, uint32_t n_new, cudaStream_t st)
{
    const uint64_t W_old = tn_row_words(n_old), W_new = tn_row_words(n_new);
    if (S_old == S_new) {
        // in place: the new columns of the old rows, then the new rows
        const uint64_t w0 = (n_old / 64) & ~1ull;
        if (n_old > 0 && w0 < W_new) {
            tn_internal_count_launches(1);
            grow_kernel<<<grow_blocks((uint64_t)n_old * ((W_new - w0) / 2)), 256, 0, st>>>(S_old, W_old, n_old, S_new,
                                                                                           W_new, 0, n_old, w0);
        }
        if (n_new > n_old) {
            tn_internal_count_launches(1);
            grow_kernel<<<grow_blocks((uint64_t)(n_new - n_old) * (W_new / 2)), 256, 0, st>>>(
                S_old, W_old, n_old, S_new, W_new, n_old, n_new, 0);
        }
    } else if (n_new > 0) {
        tn_internal_count_launches(1);
        grow_kernel<<<grow_blocks((uint64_t)n_new * (W_new / 2)), 256, 0, st>>>(S_old, W_old, n_old, S_new, W_new, 0,
                                                                               n_new, 0);
    }
    TN_CUDA_TRY(cudaGetLastError());
    return TN_OK;
}

// ---------------------------------------------------------------------------
// batch scan: validation (Section 2.1) and the start of the last timestamp group
// ---------------------------------------------------------------------------
struct ScanOut {
    unsigned long long bad;   // bit 0: endpoint >= n, bit 1: timestamps decrease
    unsigned long long last;  // first index e with t[e] == t[m-1] (sorted batches)
    long long t_first, t_last;
    long long t_before;       // largest timestamp below t[m-1] (the group before the last)
};

__global__ void scan_kernel(const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t m, uint32_t n,
                            ScanOut *out)
{
    const int64_t tl = t[m - 1];
    uint32_t bad = 0;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x) {
        if (u[e] >= n || v[e] >= n) bad |= 1u;
        if (e > 0 && t[e] < t[e - 1]) bad |= 2u;
        if (t[e] == tl && (e == 0 || t[e - 1] != tl)) atomicMin(&out->last, (unsigned long long)e);
        if (t[e] < tl) atomicMax(&out->t_before, (long long)t[e]);
    }
    if (bad) atomicOr(&out->bad, (unsigned long long)bad);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out->t_first = t[0];
        out->t_last = tl;
    }
}

template <typename T>
cudaError_t alloc_async(T **p, uint64_t count, cudaStream_t st)
{
    return cudaMallocAsync((void **)p, (count ? count : 1) * sizeof(T), st);
}

}  // namespace

// ---------------------------------------------------------------------------
// tn_grow_matrix
// ---------------------------------------------------------------------------
extern "C" tn_status tn_grow_matrix(const uint64_t *S_old, uint32_t n_old, uint64_t *S_new, uint32_t n_new,
                                    void *stream)
{
    if (!S_new || n_new < n_old || n_new >= (1u << 30) || (n_old > 0 && !S_old)) return TN_EINVAL;
    const uint64_t bytes_old = (uint64_t)n_old * tn_row_words(n_old) * 8;
    const uint64_t bytes_new = (uint64_t)n_new * tn_row_words(n_new) * 8;
    if (n_old > 0 && S_old == S_new) {
        if (tn_row_words(n_old) != tn_row_words(n_new)) return TN_EINVAL;
    } else if (n_old > 0) {
        const uintptr_t a0 = (uintptr_t)S_old, a1 = a0 + bytes_old;
        const uintptr_t b0 = (uintptr_t)S_new, b1 = b0 + bytes_new;
        if (a0 < b1 && b0 < a1) return TN_EINVAL;  // partial overlap
    }
    if (((uintptr_t)S_new & 15u) || ((uintptr_t)S_old & 15u)) return TN_EINVAL;
    return launch_grow(n_old ? S_old : nullptr, n_old, S_new, n_new, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// tn_online
// ---------------------------------------------------------------------------
struct tn_online {
    int device;
    uint32_t n;        // nodes (rows and columns)
    uint32_t row_cap;  // rows allocated: growth within the same row stride stays in place
    uint64_t *S;
    tn_plan_options opt;
    int32_t error;      // sticky: first error of an applied batch
    int has_applied;
    int64_t t_applied;  // last timestamp applied to S
    // pending (held-back) last timestamp group
    uint32_t *pu, *pv;
    int64_t *pt;
    uint64_t pending, pending_cap;
    int64_t pending_t;
    // concatenation of the pending group and a new batch
    uint32_t *wu, *wv;
    int64_t *wt;
    uint64_t work_cap;
    ScanOut *scan;
    tn_plan *inflight;  // plan of the last applied batch, released at the next call
    uint64_t applied_events, batches;
    // two-stream mode (tn::online_use_apply_stream): the matrix updates run on
    // `ast` while copies and scheduling run on the caller's stream; the plans
    // of applied batches are released once an event behind their update has
    // completed, without waiting for it
    cudaStream_t ast;
    int32_t *dstatus;  // status word shared by every batch's plan (device)
    tn_plan *flight[tn::kOnlineFlight];
    cudaEvent_t flight_done[tn::kOnlineFlight];
    uint32_t flight_head, flight_count;
};

namespace {

uint32_t rows_for(uint32_t n)
{
    const uint64_t r = ((uint64_t)n + 1023) / 1024 * 1024;
    return (uint32_t)(r < (1u << 30) ? r : (1u << 30) - 1);
}

bool on_device(const tn_online *o)
{
    int dev = -1;
    return cudaGetDevice(&dev) == cudaSuccess && dev == o->device;
}

// Two-stream mode: releases the plans of applied batches whose update has
// finished (all of them, waiting, with `wait`), folding their status into the
// sticky error.
tn_status reap(tn_online *o, bool wait)
{
    while (o->flight_count > 0) {
        const uint32_t i = o->flight_head;
        if (wait) {
            cudaEventSynchronize(o->flight_done[i]);
        } else {
            const cudaError_t q = cudaEventQuery(o->flight_done[i]);
            if (q == cudaErrorNotReady) break;
        }
        // the plans share o->dstatus, read once by tn_online_status
        tn_plan_destroy(o->flight[i], o->ast);
        cudaEventDestroy(o->flight_done[i]);
        o->flight_head = (i + 1) % tn::kOnlineFlight;
        o->flight_count--;
    }
    return (tn_status)o->error;
}

// Waits for the last applied batch and folds its status into the sticky error.
tn_status settle(tn_online *o, cudaStream_t st)
{
    if (o->ast) {
        reap(o, true);
        int32_t h = 0;
        cudaError_t err = cudaMemcpyAsync(&h, o->dstatus, sizeof(h), cudaMemcpyDeviceToHost, o->ast);
        if (err == cudaSuccess) err = tn_internal_stream_wait(o->ast);
        if (err != cudaSuccess) h = TN_ECUDA;
        if (h != TN_OK && o->error == TN_OK) o->error = h;
        return (tn_status)o->error;
    }
    if (o->inflight) {
        const tn_status rc = tn_plan_status(o->inflight, st);
        tn_plan_destroy(o->inflight, st);
        o->inflight = nullptr;
        if (rc != TN_OK && o->error == TN_OK) o->error = rc;
    }
    return (tn_status)o->error;
}

template <typename T>
tn_status ensure(T **buf, uint64_t *cap_unused, uint64_t need, uint64_t keep, cudaStream_t st)
{
    (void)cap_unused;
    T *fresh = nullptr;
    TN_CUDA_TRY(alloc_async(&fresh, need, st));
    if (*buf && keep) {
        cudaError_t err = cudaMemcpyAsync(fresh, *buf, keep * sizeof(T), cudaMemcpyDeviceToDevice, st);
        if (err != cudaSuccess) {
            cudaFreeAsync(fresh, st);
            tn_internal_set_cuda_error(err);
            return TN_ECUDA;
        }
    }
    if (*buf) cudaFreeAsync(*buf, st);
    *buf = fresh;
    return TN_OK;
}

// Room for `need` pending events, keeping the first `keep`.
tn_status reserve_pending(tn_online *o, uint64_t need, uint64_t keep, cudaStream_t st)
{
    if (need <= o->pending_cap) return TN_OK;
    uint64_t cap = o->pending_cap ? o->pending_cap : 1024;
    while (cap < need) cap *= 2;
    tn_status rc = ensure(&o->pu, nullptr, cap, keep, st);
    if (rc == TN_OK) rc = ensure(&o->pv, nullptr, cap, keep, st);
    if (rc == TN_OK) rc = ensure(&o->pt, nullptr, cap, keep, st);
    if (rc == TN_OK) o->pending_cap = cap;
    return rc;
}

tn_status reserve_work(tn_online *o, uint64_t need, cudaStream_t st)
{
    if (need <= o->work_cap) return TN_OK;
    uint64_t cap = o->work_cap ? o->work_cap : 4096;
    while (cap < need) cap *= 2;
    tn_status rc = ensure(&o->wu, nullptr, cap, 0, st);
    if (rc == TN_OK) rc = ensure(&o->wv, nullptr, cap, 0, st);
    if (rc == TN_OK) rc = ensure(&o->wt, nullptr, cap, 0, st);
    if (rc == TN_OK) o->work_cap = cap;
    return rc;
}

// Schedules and applies `count` complete timestamp groups to S.
tn_status apply_ready(tn_online *o, const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t count,
                      cudaStream_t st)
{
    tn_plan *plan = nullptr;
    // two-stream mode: the update waits for the plan's last kernels through an
    // event on the apply stream instead of a host wait
    tn_status rc = o->ast ? tn::plan_create_ordered(u, v, t, count, o->n, &o->opt, st, &plan)
                          : tn_plan_create(u, v, t, count, o->n, nullptr, &o->opt, st, &plan);
    if (rc != TN_OK) return rc;
    if (o->ast) {
        rc = tn::plan_use_status(plan, o->dstatus, st);
        cudaEvent_t planned = nullptr;
        cudaError_t perr = cudaEventCreateWithFlags(&planned, cudaEventDisableTiming);
        if (perr == cudaSuccess) perr = cudaEventRecord(planned, st);
        if (perr == cudaSuccess) perr = cudaStreamWaitEvent(o->ast, planned, 0);
        if (planned) cudaEventDestroy(planned);  // released once it has completed
        if (perr != cudaSuccess) {
            tn_internal_set_cuda_error(perr);
            rc = TN_ECUDA;
        }
        if (rc != TN_OK) {
            tn_plan_destroy(plan, st);  // behind the kernels that write it
            return rc;
        }
        // the plan is complete (tn_plan_create returned), so the update may run
        // on the apply stream behind the earlier ones
        if (o->flight_count == tn::kOnlineFlight) {  // room in the ring: wait for the oldest update
            cudaEventSynchronize(o->flight_done[o->flight_head]);
            reap(o, false);
        }
        cudaEvent_t done = nullptr;
        cudaError_t err = cudaEventCreateWithFlags(&done, cudaEventBlockingSync | cudaEventDisableTiming);
        if (err == cudaSuccess) {
            rc = tn_plan_apply(plan, o->S, o->n, nullptr, nullptr, 0u, o->ast);
            if (rc == TN_OK) err = cudaEventRecord(done, o->ast);
        }
        if (err != cudaSuccess || rc != TN_OK) {
            if (done) cudaEventDestroy(done);
            tn_plan_destroy(plan, o->ast);
            if (err != cudaSuccess) {
                tn_internal_set_cuda_error(err);
                return TN_ECUDA;
            }
            return rc;
        }
        const uint32_t slot = (o->flight_head + o->flight_count) % tn::kOnlineFlight;
        o->flight[slot] = plan;
        o->flight_done[slot] = done;
        o->flight_count++;
        o->applied_events += count;
        return TN_OK;
    }
    rc = tn_plan_apply(plan, o->S, o->n, nullptr, nullptr, 0u, st);
    if (rc != TN_OK) {
        tn_plan_destroy(plan, st);
        return rc;
    }
    o->inflight = plan;
    o->applied_events += count;
    return TN_OK;
}

tn_status copy_events(uint32_t *du, uint32_t *dv, int64_t *dt, const uint32_t *u, const uint32_t *v,
                      const int64_t *t, uint64_t count, cudaStream_t st)
{
    if (!count) return TN_OK;
    TN_CUDA_TRY(cudaMemcpyAsync(du, u, count * 4, cudaMemcpyDeviceToDevice, st));
    TN_CUDA_TRY(cudaMemcpyAsync(dv, v, count * 4, cudaMemcpyDeviceToDevice, st));
    TN_CUDA_TRY(cudaMemcpyAsync(dt, t, count * 8, cudaMemcpyDeviceToDevice, st));
    return TN_OK;
}

}  // namespace

extern "C" tn_status tn_online_create(uint32_t n, const tn_plan_options *opt, void *stream, tn_online **out)
{
    if (!out) return TN_EINVAL;
    *out = nullptr;
    if (n == 0 || n >= (1u << 30)) return TN_EINVAL;
    if (opt) {
        for (int i = 0; i < 2; ++i)
            if (opt->reserved[i]) return TN_EINVAL;
        if (opt->directed > 1 || opt->resident_words) return TN_EINVAL;
        const uint32_t sw = opt->slab_words;
        if (sw && (sw < 2 || sw > tn::kMaxSlabWords || (sw & 1u))) return TN_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    tn_internal_keep_pool();
    tn_online *o = (tn_online *)calloc(1, sizeof(tn_online));
    if (!o) return TN_ENOMEM;
    if (opt) o->opt = *opt;
    cudaGetDevice(&o->device);
    o->n = n;
    o->row_cap = rows_for(n);
    tn_status rc = TN_OK;
    cudaError_t err = alloc_async(&o->S, (uint64_t)o->row_cap * tn_row_words(n), st);
    if (err == cudaSuccess) err = alloc_async(&o->scan, 1, st);
    if (err != cudaSuccess) {
        tn_internal_set_cuda_error(err);
        rc = err == cudaErrorMemoryAllocation ? TN_ENOMEM : TN_ECUDA;
    }
    if (rc == TN_OK) rc = tn_init_matrix(o->S, n, n, nullptr, stream);
    if (rc != TN_OK) {
        if (o->S) cudaFreeAsync(o->S, st);
        if (o->scan) cudaFreeAsync(o->scan, st);
        free(o);
        return rc;
    }
    *out = o;
    return TN_OK;
}

extern "C" tn_status tn_online_push(tn_online *o, const uint32_t *u, const uint32_t *v, const int64_t *t,
                                    uint64_t m, uint32_t flags, void *stream)
{
    if (!o || (flags & ~TN_GROUP_END) || !on_device(o)) return TN_EINVAL;
    if (m > 0 && (!u || !v || !t)) return TN_EINVAL;
    if (m >= (1ull << 30) || o->pending + m >= (1ull << 30)) return TN_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    tn_status rc = o->ast ? reap(o, false) : settle(o, st);
    if (rc != TN_OK) return rc;

    const uint64_t P = o->pending;  // events held back from the previous batch
    uint64_t g;                     // the first g events of (pending ++ batch) are complete groups
    int64_t t_end, t_before = 0;  // last timestamp; timestamp of the group before it
    if (m == 0) {
        if (!(flags & TN_GROUP_END) || P == 0) return TN_OK;
        g = P;
        t_end = o->pending_t;
    } else {
        ScanOut init;
        init.bad = 0;
        init.last = ~0ull;
        init.t_first = init.t_last = 0;
        init.t_before = INT64_MIN;
        ScanOut res;
        TN_CUDA_TRY(cudaMemcpyAsync(o->scan, &init, sizeof(init), cudaMemcpyHostToDevice, st));
        const uint64_t b = (m + 255) / 256;
        tn_internal_count_launches(1);
        scan_kernel<<<(int)(b < 1216 ? b : 1216), 256, 0, st>>>(u, v, t, m, o->n, o->scan);
        TN_CUDA_TRY(cudaGetLastError());
        TN_CUDA_TRY(cudaMemcpyAsync(&res, o->scan, sizeof(res), cudaMemcpyDeviceToHost, st));
        TN_CUDA_TRY(tn_internal_stream_wait(st));
        if (res.bad & 1ull) return TN_ERANGE;
        if (res.bad & 2ull) return TN_EORDER;
        if (P > 0 ? res.t_first < o->pending_t : (o->has_applied && res.t_first <= o->t_applied)) return TN_EORDER;
        t_end = res.t_last;
        t_before = res.t_before;
        if (flags & TN_GROUP_END)
            g = P + m;
        else if (res.last > 0)
            g = P + res.last;
        else  // the whole batch is one group: it continues the pending one or follows it
            g = (P > 0 && res.t_first == o->pending_t) ? 0 : P;
    }
    const uint64_t M = P + m;

    // 1. apply the complete groups
    if (g > 0) {
        if (P == 0) {
            rc = apply_ready(o, u, v, t, g, st);
        } else if (g == P) {
            rc = apply_ready(o, o->pu, o->pv, o->pt, g, st);
        } else {
            rc = reserve_work(o, g, st);
            if (rc == TN_OK) rc = copy_events(o->wu, o->wv, o->wt, o->pu, o->pv, o->pt, P, st);
            if (rc == TN_OK) rc = copy_events(o->wu + P, o->wv + P, o->wt + P, u, v, t, g - P, st);
            if (rc == TN_OK) rc = apply_ready(o, o->wu, o->wv, o->wt, g, st);
        }
        if (rc != TN_OK) return rc;  // nothing was applied: the state is unchanged
        o->has_applied = 1;
        o->t_applied = g == M ? t_end : g == P ? o->pending_t : t_before;
    }

    // 2. hold back the rest (the last group, possibly continued later)
    if (g < M) {
        if (g >= P) {
            // the pending events now come from the batch only; the old ones were applied
            // (stream order puts these copies after the plan has read them)
            rc = reserve_pending(o, M - g, 0, st);
            if (rc == TN_OK) rc = copy_events(o->pu, o->pv, o->pt, u + (g - P), v + (g - P), t + (g - P), M - g, st);
        } else {
            // g == 0: the whole batch continues the pending group
            rc = reserve_pending(o, M, P, st);
            if (rc == TN_OK) rc = copy_events(o->pu + P, o->pv + P, o->pt + P, u, v, t, m, st);
        }
        if (rc != TN_OK) {
            if (o->error == TN_OK) o->error = rc;  // the state is no longer consistent
            return rc;
        }
        o->pending = M - g;
        o->pending_t = t_end;
    } else {
        o->pending = 0;
    }
    o->batches += 1;
    return TN_OK;
}

extern "C" tn_status tn_online_flush(tn_online *o, void *stream)
{
    return tn_online_push(o, nullptr, nullptr, nullptr, 0, TN_GROUP_END, stream);
}

extern "C" tn_status tn_online_grow(tn_online *o, uint32_t n_new, void *stream)
{
    if (!o || n_new < o->n || n_new >= (1u << 30) || !on_device(o)) return TN_EINVAL;
    cudaStream_t st = o->ast ? o->ast : (cudaStream_t)stream;  // the matrix lives on the apply stream
    tn_status rc = o->ast ? reap(o, false) : settle(o, st);
    if (rc != TN_OK) return rc;
    if (n_new == o->n) return TN_OK;
    if (tn_row_words(n_new) == tn_row_words(o->n) && n_new <= o->row_cap) {
        rc = launch_grow(o->S, o->n, o->S, n_new, st);
        if (rc != TN_OK) return rc;
    } else {
        const uint32_t cap = rows_for(n_new);
        uint64_t *fresh = nullptr;
        TN_CUDA_TRY(alloc_async(&fresh, (uint64_t)cap * tn_row_words(n_new), st));
        rc = launch_grow(o->S, o->n, fresh, n_new, st);
        if (rc != TN_OK) {
            cudaFreeAsync(fresh, st);
            return rc;
        }
        cudaFreeAsync(o->S, st);
        o->S = fresh;
        o->row_cap = cap;
    }
    o->n = n_new;
    return TN_OK;
}

tn_status tn::online_use_apply_stream(tn_online *o, cudaStream_t apply_stream)
{
    if (!o || !apply_stream || o->ast || o->batches || o->inflight) return TN_EINVAL;
    TN_CUDA_TRY(cudaMallocAsync((void **)&o->dstatus, sizeof(int32_t), apply_stream));
    TN_CUDA_TRY(cudaMemsetAsync(o->dstatus, 0, sizeof(int32_t), apply_stream));
    o->ast = apply_stream;
    return TN_OK;
}

const int32_t *tn::online_status_word(const tn_online *o) { return o ? o->dstatus : nullptr; }

extern "C" tn_status tn_online_status(tn_online *o, void *stream)
{
    if (!o) return TN_EINVAL;
    return settle(o, (cudaStream_t)stream);
}

extern "C" tn_status tn_online_get_state(const tn_online *o, tn_online_state *s)
{
    if (!o || !s) return TN_EINVAL;
    memset(s, 0, sizeof(*s));
    s->S = o->S;
    s->n = o->n;
    s->row_words = tn_row_words(o->n);
    s->pending_events = o->pending;
    s->pending_t = o->pending_t;
    s->applied_events = o->applied_events;
    s->batches = o->batches;
    s->has_applied = (uint32_t)o->has_applied;
    s->t_applied = o->t_applied;
    return TN_OK;
}

extern "C" tn_status tn_online_destroy(tn_online *o, void *stream)
{
    if (!o) return TN_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (o->ast) reap(o, true);
    if (o->inflight) tn_plan_destroy(o->inflight, st);
    if (o->dstatus) cudaFreeAsync(o->dstatus, o->ast);
    cudaFreeAsync(o->S, o->ast ? o->ast : st);
    cudaFreeAsync(o->scan, st);
    if (o->pu) cudaFreeAsync(o->pu, st);
    if (o->pv) cudaFreeAsync(o->pv, st);
    if (o->pt) cudaFreeAsync(o->pt, st);
    if (o->wu) cudaFreeAsync(o->wu, st);
    if (o->wv) cudaFreeAsync(o->wv, st);
    if (o->wt) cudaFreeAsync(o->wt, st);
    free(o);
    return TN_OK;
}
