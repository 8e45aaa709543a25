// Batched application under a CUDA graph, and the launch-shape autotuner.
//
// Network hashing (Section 4.2) builds R proxy component matrices from R
// proxy event streams of the same length; many networks of different n and m
// can share one launch of the streaming kernel (tn_plan_apply_batch).  The
// whole batched step (initialisation, order gates, the persistent streaming
// launch) is captured once into a CUDA graph and replayed with one launch.
//
// The autotuner picks the plan options that decide the launch shape -- slab
// width (columns per CTA, hence the CTA count), scheduling-window depth, the
// size of the shared-memory row buffer (hence CTAs per SM), or the
// resident-slab form for small networks -- by timing the candidates (their
// schedule and their application) on a prefix of the events, for a batch of
// `replicas` networks of the same size, and caches the choice per (device, n,
// ncols, replicas, log2 m).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <chrono>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "tn_internal.cuh"

struct tn_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t launches = 0;  // kernels per replay
};

extern "C" tn_status tn_graph_capture_batch(const tn_plan *const *plans, uint64_t *const *S, const uint32_t *ncols,
                                            uint32_t count, uint32_t flags, tn_graph **out)
{
    if (!plans || !S || !ncols || count == 0 || !out || (flags & ~TN_INIT_IDENTITY)) return TN_EINVAL;
    *out = nullptr;
    tn_graph *g = new (std::nothrow) tn_graph();
    if (!g) return TN_ENOMEM;
    cudaStream_t cs = nullptr;
    cudaError_t err = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (err != cudaSuccess) {
        delete g;
        tn_internal_set_cuda_error(err);
        return TN_ECUDA;
    }
    std::vector<const uint32_t *> src(count, nullptr);
    const uint64_t before = tn_kernel_launches();
    err = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    tn_status rc = TN_OK;
    if (err == cudaSuccess) {
        rc = tn::apply_jobs(plans, S, ncols, src.data(), nullptr, count, flags, cs);
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        g->graph = graph;
        if (rc == TN_OK && e2 != cudaSuccess) {
            err = e2;
            rc = TN_ECUDA;
        }
    } else {
        rc = TN_ECUDA;
    }
    if (rc == TN_OK) {
        err = cudaGraphInstantiate(&g->exec, g->graph, 0);
        if (err != cudaSuccess) rc = TN_ECUDA;
    }
    g->launches = tn_kernel_launches() - before;
    cudaStreamDestroy(cs);
    if (rc != TN_OK) {
        if (err != cudaSuccess) tn_internal_set_cuda_error(err);
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return rc;
    }
    *out = g;
    return TN_OK;
}

extern "C" tn_status tn_graph_launch(tn_graph *g, void *stream)
{
    if (!g || !g->exec) return TN_EINVAL;
    TN_CUDA_TRY(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    tn_internal_count_launches(g->launches);
    return TN_OK;
}

extern "C" tn_status tn_graph_destroy(tn_graph *g)
{
    if (!g) return TN_EINVAL;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return TN_OK;
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
namespace {

std::mutex g_tune_mu;
std::map<std::tuple<int, uint32_t, uint32_t, uint32_t, int>, tn_tune_result> g_tune_cache;

constexpr uint64_t kTuneBytesCap = 64ull << 30;  // scratch matrices of one timing run: at most this,
                                                 // and at most half of the free device memory
constexpr uint32_t kTuneWidest = 64;             // widest slab tried

// Time of one batched application of `plan` to `count` matrices of `ncols`
// columns (the first ncols node ids as sources when ncols < n), best of 2.
tn_status time_apply(tn_plan *plan, uint64_t *const *mats, uint32_t count, uint32_t ncols, const uint32_t *src,
                     cudaStream_t st, float *ms)
{
    cudaEvent_t e0, e1;
    TN_CUDA_TRY(cudaEventCreate(&e0));
    TN_CUDA_TRY(cudaEventCreate(&e1));
    float best = INFINITY;
    tn_status rc = TN_OK;
    for (int rep = 0; rep < 2 && rc == TN_OK; ++rep) {
        cudaEventRecord(e0, st);
        for (uint32_t r = 0; r < count && rc == TN_OK; ++r)
            if (src) rc = tn_init_matrix(mats[r], plan->n, ncols, src, st);
        std::vector<const tn_plan *> plans(count, plan);
        std::vector<uint32_t> nc(count, ncols);
        if (rc == TN_OK)
            rc = tn_plan_apply_batch(plans.data(), mats, nc.data(), nullptr, count, src ? 0u : TN_INIT_IDENTITY, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = TN_ECUDA;
        float t = 0.f;
        if (rc == TN_OK && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess && t < best) best = t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return rc;
}

// tn_plan_create on the sample, with its wall time (the planner synchronises
// with the host, so this is its whole cost).
tn_status timed_plan(const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t m, uint32_t n,
                     const tn_plan_options *opt, cudaStream_t st, tn_plan **plan, float *ms)
{
    TN_CUDA_TRY(cudaStreamSynchronize(st));
    const auto t0 = std::chrono::steady_clock::now();
    const tn_status rc = tn_plan_create(u, v, t, m, n, nullptr, opt, st, plan);
    *ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}

}  // namespace

// The full problem (replicas x ceil(row words / slab) CTAs) runs in waves of
// SMs x CTAs-per-SM; every candidate is timed on one wave's worth of CTAs --
// whole matrices for small networks, a subset of source columns for large ones
// (columns are independent, so a CTA's work does not depend on the others) --
// and scored as waves x that time plus replicas x the schedule's build time
// on the sample (each application of a plan is preceded by building it).
extern "C" tn_status tn_autotune(const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t m, uint32_t n,
                                 uint32_t ncols_full, uint32_t replicas, uint64_t sample_events, void *stream,
                                 tn_tune_result *out)
{
    if (ncols_full == 0) ncols_full = n;
    if (!u || !v || !t || m == 0 || n == 0 || n >= (1u << 30) || replicas == 0 || replicas > 64 || !out ||
        ncols_full > n)
        return TN_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    TN_CUDA_TRY(cudaGetDevice(&dev));
    TN_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int mb = (int)floor(log2((double)m));
    const auto key = std::make_tuple(dev, n, ncols_full, replicas, mb);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *out = it->second;
            out->cached = 1;
            return TN_OK;
        }
    }
    memset(out, 0, sizeof(*out));
    const uint64_t ld = tn_row_words(ncols_full);
    const uint64_t msample = sample_events && sample_events < m ? sample_events : m;
    out->sample_events = msample;

    size_t free_b = 0, total_b = 0;
    TN_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    const uint64_t kTuneBytesLimit = free_b / 2 < kTuneBytesCap ? free_b / 2 : kTuneBytesCap;
    // source ids 0..max-1 for column-subset timings
    const uint32_t max_cols = (uint32_t)nsm * 2u * kTuneWidest * 64u;
    uint32_t *ids = nullptr;
    std::vector<uint32_t> hids(max_cols);
    for (uint32_t i = 0; i < max_cols; ++i) hids[i] = i;
    TN_CUDA_TRY(cudaMallocAsync((void **)&ids, max_cols * sizeof(uint32_t), st));
    TN_CUDA_TRY(cudaMemcpyAsync(ids, hids.data(), max_cols * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    TN_CUDA_TRY(cudaStreamSynchronize(st));

    // slabs above 16 words (256- to 512-byte row segments, 192 KB row buffer)
    // suit large networks whose windows stream from global memory; they run one
    // CTA per SM
    const uint32_t slabs[] = {2, 4, 8, 12, 16, 24, 32, 48, kTuneWidest};
    const uint32_t windows[] = {320, 640, 1024};
    float best = INFINITY;
    tn_status rc = TN_OK;
    for (uint32_t sw : slabs) {
        if (sw > ld || rc != TN_OK) continue;
        for (int half = 0; half < (sw <= 16 ? 2 : 1) && rc == TN_OK; ++half) {
            const uint64_t occ = half ? 2 : 1;  // 32 KB of stages + 80 or 160 (192) KB of rows per CTA
            const uint64_t per_rep = (ld + sw - 1) / sw;
            const uint64_t total = per_rep * replicas;
            const uint64_t slots = (uint64_t)nsm * occ;
            const uint64_t waves = (total + slots - 1) / slots;
            // one wave's worth of CTAs
            uint32_t reps = 1, ncols = ncols_full;
            const uint32_t *src = ncols_full < n ? ids : nullptr;
            if (per_rep >= slots) {
                uint64_t c = slots;
                while (c > 1 && (uint64_t)n * tn_row_words(c * sw * 64) * 8 > kTuneBytesLimit) c /= 2;
                if (c * sw * 64 < ncols_full) {
                    ncols = (uint32_t)(c * sw * 64);
                    src = ids;
                }
            } else {
                reps = (uint32_t)((slots + per_rep - 1) / per_rep);
                if (reps > replicas) reps = replicas;
                while (reps > 1 && (uint64_t)reps * n * ld * 8 > kTuneBytesLimit) --reps;
                if ((uint64_t)n * ld * 8 > kTuneBytesLimit) continue;
                if (src && ncols > max_cols) continue;
            }
            std::vector<uint64_t *> mats(reps, nullptr);
            const uint64_t mbytes = (uint64_t)n * tn_row_words(ncols) * 8;
            for (uint32_t r = 0; r < reps && rc == TN_OK; ++r) {
                const cudaError_t e = cudaMallocAsync((void **)&mats[r], mbytes, st);
                if (e != cudaSuccess) {
                    tn_internal_set_cuda_error(e);
                    rc = e == cudaErrorMemoryAllocation ? TN_ENOMEM : TN_ECUDA;
                }
            }
            for (uint32_t win : windows) {
                if (rc != TN_OK) break;
                tn_plan_options opt;
                memset(&opt, 0, sizeof(opt));
                opt.window_events = win;
                opt.slab_words = sw;
                opt.smem_rows = (half ? 80u : (sw <= 16 ? 160u : 192u)) * 1024u / (8u * sw);
                tn_plan *plan = nullptr;
                float pms = 0.f;
                rc = timed_plan(u, v, t, msample, n, &opt, st, &plan, &pms);
                if (rc != TN_OK) break;
                float tms = INFINITY;
                rc = time_apply(plan, mats.data(), reps, ncols, src, st, &tms);
                if (rc == TN_OK) rc = tn_plan_status(plan, st);
                tn_plan_destroy(plan, st);
                if (rc != TN_OK) break;
                out->tried++;
                const float score = tms * (float)waves + pms * (float)replicas;
                if (score < best) {
                    best = score;
                    out->best = opt;
                    out->best_ms = score;
                }
            }
            for (uint64_t *p : mats)
                if (p) cudaFreeAsync(p, st);
        }
    }
    // the resident-slab form, for networks whose rows fit shared memory: one
    // CTA per resident_words words of the row, one CTA per SM beyond a wave
    // unless two fit (the launch's rule); a plan whose saved rows do not fit
    // is skipped
    const uint32_t rws[] = {1, 2};
    const uint64_t used_words = (ncols_full + 63) / 64;
    for (uint32_t rw : rws) {
        if (rc != TN_OK || n > tn::resident_max_rows(rw)) continue;
        const uint64_t per_rep = (used_words + rw - 1) / rw;
        const uint64_t total = per_rep * replicas;
        const uint64_t rb = 128 + (((uint64_t)n * 8 * rw + 127) & ~127ull);
        const uint64_t occ = (total > (uint64_t)nsm && rb + 2ull * 16384 <= 112ull * 1024) ? 2 : 1;
        const uint64_t slots = (uint64_t)nsm * occ;
        const uint64_t waves = (total + slots - 1) / slots;
        uint32_t reps = 1, ncols = ncols_full;
        const uint32_t *src = ncols_full < n ? ids : nullptr;
        if (per_rep >= slots) {
            const uint64_t c = slots * rw * 64;
            if (c < ncols_full) {
                ncols = (uint32_t)c;
                src = ids;
            }
        } else {
            reps = (uint32_t)((slots + per_rep - 1) / per_rep);
            if (reps > replicas) reps = replicas;
            while (reps > 1 && (uint64_t)reps * n * ld * 8 > kTuneBytesLimit) --reps;
        }
        if (src && ncols > max_cols) continue;
        std::vector<uint64_t *> mats(reps, nullptr);
        const uint64_t mbytes = (uint64_t)n * tn_row_words(ncols) * 8;
        for (uint32_t r = 0; r < reps && rc == TN_OK; ++r) {
            const cudaError_t e = cudaMallocAsync((void **)&mats[r], mbytes, st);
            if (e != cudaSuccess) {
                tn_internal_set_cuda_error(e);
                rc = e == cudaErrorMemoryAllocation ? TN_ENOMEM : TN_ECUDA;
            }
        }
        const uint32_t rwindows[] = {640, 2048};
        for (uint32_t win : rwindows) {
            if (rc != TN_OK) break;
            tn_plan_options opt;
            memset(&opt, 0, sizeof(opt));
            opt.window_events = win;
            opt.resident_words = rw;
            tn_plan *plan = nullptr;
            float pms = 0.f;
            const tn_status pc = timed_plan(u, v, t, msample, n, &opt, st, &plan, &pms);
            if (pc == TN_EINVAL) continue;  // saved rows do not fit beside the rows
            rc = pc;
            if (rc != TN_OK) break;
            float tms = INFINITY;
            rc = time_apply(plan, mats.data(), reps, ncols, src, st, &tms);
            if (rc == TN_OK) rc = tn_plan_status(plan, st);
            tn_plan_destroy(plan, st);
            if (rc != TN_OK) break;
            out->tried++;
            const float score = tms * (float)waves + pms * (float)replicas;
            if (score < best) {
                best = score;
                out->best = opt;
                out->best_ms = score;
            }
        }
        for (uint64_t *p : mats)
            if (p) cudaFreeAsync(p, st);
    }
    cudaFreeAsync(ids, st);
    if (rc != TN_OK) return rc;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = *out;
    return TN_OK;
}
