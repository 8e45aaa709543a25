// Batched application under a CUDA graph, and the launch-shape autotuner.
//
// Network hashing (Section 4.2) builds R proxy component matrices from R
// proxy event streams of the same length; many networks of different n and m
// can share one launch of the streaming kernel (tn_plan_apply_batch).  The
// whole batched step (initialisation, order gates, the persistent streaming
// launch) is captured once into a CUDA graph and replayed with one launch.
//
// The autotuner picks the plan options that decide the launch shape -- slab
// width (columns per CTA, hence the CTA count), scheduling-window depth, and
// the size of the shared-memory row buffer (hence CTAs per SM) -- by timing
// the candidates on a prefix of the events, for a batch of `replicas`
// networks of the same size, and caches the choice per (device, n, replicas,
// log2 m).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

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
std::map<std::tuple<int, uint32_t, uint32_t, int>, tn_tune_result> g_tune_cache;

constexpr uint64_t kTuneBytesLimit = 8ull << 30;  // scratch matrices of one tuning run

struct Scratch {
    std::vector<uint64_t *> mats;
    cudaStream_t st;
    ~Scratch()
    {
        for (uint64_t *p : mats)
            if (p) cudaFreeAsync(p, st);
    }
};

// Time of one batched application of `plan` to every scratch matrix (best of 2).
tn_status time_apply(tn_plan *plan, const Scratch &sc, uint32_t n, cudaStream_t st, float *ms)
{
    const uint32_t count = (uint32_t)sc.mats.size();
    std::vector<const tn_plan *> plans(count, plan);
    std::vector<uint32_t> ncols(count, n);
    cudaEvent_t e0, e1;
    TN_CUDA_TRY(cudaEventCreate(&e0));
    TN_CUDA_TRY(cudaEventCreate(&e1));
    float best = INFINITY;
    tn_status rc = TN_OK;
    for (int rep = 0; rep < 2 && rc == TN_OK; ++rep) {
        cudaEventRecord(e0, st);
        rc = tn_plan_apply_batch(plans.data(), sc.mats.data(), ncols.data(), count, TN_INIT_IDENTITY, st);
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

}  // namespace

extern "C" tn_status tn_autotune(const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t m, uint32_t n,
                                 uint32_t replicas, uint64_t sample_events, void *stream, tn_tune_result *out)
{
    if (!u || !v || !t || m == 0 || n == 0 || n >= (1u << 30) || replicas == 0 || replicas > 64 || !out)
        return TN_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    TN_CUDA_TRY(cudaGetDevice(&dev));
    const int mb = (int)floor(log2((double)m));
    const auto key = std::make_tuple(dev, n, replicas, mb);
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
    const uint64_t ld = tn_row_words(n);
    const uint64_t ms = sample_events && sample_events < m ? sample_events : m;
    out->sample_events = ms;
    if ((uint64_t)replicas * n * ld * 8 > kTuneBytesLimit) {
        // too large to time here: keep the defaults
        return TN_OK;
    }
    Scratch sc;
    sc.st = st;
    for (uint32_t r = 0; r < replicas; ++r) {
        uint64_t *p = nullptr;
        TN_CUDA_TRY(cudaMallocAsync((void **)&p, (size_t)n * ld * 8, st));
        sc.mats.push_back(p);
    }
    const uint32_t slabs[] = {2, 4, 8, 12, 16};
    const uint32_t windows[] = {320, 640, 1024};
    float best = INFINITY;
    for (uint32_t sw : slabs) {
        if (sw > ld) continue;
        for (uint32_t win : windows) {
            for (int half = 0; half < 2; ++half) {
                tn_plan_options opt;
                memset(&opt, 0, sizeof(opt));
                opt.window_events = win;
                opt.slab_words = sw;
                opt.smem_rows = (half ? 80u : 160u) * 1024u / (8u * sw);
                tn_plan *plan = nullptr;
                tn_status rc = tn_plan_create(u, v, t, ms, n, nullptr, &opt, st, &plan);
                if (rc != TN_OK) return rc;
                float tms = INFINITY;
                rc = time_apply(plan, sc, n, st, &tms);
                if (rc == TN_OK) rc = tn_plan_status(plan, st);
                tn_plan_destroy(plan, st);
                if (rc != TN_OK) return rc;
                out->tried++;
                if (tms < best) {
                    best = tms;
                    out->best = opt;
                    out->best_ms = tms;
                }
            }
        }
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = *out;
    return TN_OK;
}
