// Status strings, layout helper and the host-buffer end-to-end entry point.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tn_internal.cuh"

// Last CUDA runtime error seen by a libtn call on this thread (diagnostics).
static thread_local cudaError_t g_last_cuda_error = cudaSuccess;

void tn_internal_set_cuda_error(cudaError_t err) { g_last_cuda_error = err; }

extern "C" const char *tn_last_cuda_error(void) { return cudaGetErrorString(g_last_cuda_error); }

#include <atomic>
#include <mutex>

void tn_internal_keep_pool(void)
{
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    done[dev] = true;
}
cudaError_t tn_internal_stream_wait(cudaStream_t st)
{
    struct Cached {
        int dev = -1;
        cudaEvent_t ev = nullptr;
        ~Cached()
        {
            if (ev) cudaEventDestroy(ev);
        }
    };
    thread_local Cached c;
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (c.dev != dev) {
        if (c.ev) cudaEventDestroy(c.ev);
        c.ev = nullptr;
        err = cudaEventCreateWithFlags(&c.ev, cudaEventBlockingSync | cudaEventDisableTiming);
        if (err != cudaSuccess) return err;
        c.dev = dev;
    }
    err = cudaEventRecord(c.ev, st);
    if (err != cudaSuccess) return err;
    return cudaEventSynchronize(c.ev);
}

cudaError_t tn_internal_allow_max_dyn_smem(const void *kernel)
{
    int dev = 0, optin = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (err == cudaSuccess) err = cudaFuncGetAttributes(&fa, kernel);
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return err;
}

static std::atomic<uint64_t> g_launches{0};
void tn_internal_count_launches(uint64_t count) { g_launches.fetch_add(count, std::memory_order_relaxed); }
extern "C" uint64_t tn_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" const char *tn_status_string(tn_status s)
{
    switch (s) {
    case TN_OK: return "TN_OK";
    case TN_EINVAL: return "TN_EINVAL: invalid argument";
    case TN_ERANGE: return "TN_ERANGE: node id out of range";
    case TN_EORDER: return "TN_EORDER: timestamps out of order";
    case TN_ENOMEM: return "TN_ENOMEM: device allocation failed";
    case TN_ECUDA: return "TN_ECUDA: CUDA runtime error";
    case TN_ETIMEOUT: return "TN_ETIMEOUT: bounded device wait expired";
    case TN_ESCRATCH: return "TN_ESCRATCH: problem larger than the fixed scratch of a no-alloc entry point";
    default: return "unknown tn_status";
    }
}

extern "C" uint64_t tn_row_words(uint64_t ncols) { return ((ncols + 1023) / 1024) * 16; }

// Whole exact path from host arrays: H2D copy of the events, component matrix
// from the identity (Algorithm 1), out-sizes (Section 3.1), D2H copy.
extern "C" tn_status tn_out_component_sizes_host(const uint32_t *u, const uint32_t *v, const int64_t *t,
                                                 uint64_t m, uint32_t n, const tn_plan_options *opt,
                                                 uint32_t *out_sizes, uint32_t *argmax, void *stream)
{
    if (!out_sizes || n == 0 || n >= (1u << 30) || (m > 0 && (!u || !v || !t))) return TN_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    tn_internal_keep_pool();
    const uint64_t ld = tn_row_words(n);
    uint32_t *du = nullptr, *dv = nullptr, *dout = nullptr, *dam = nullptr;
    int64_t *dt = nullptr;
    uint64_t *S = nullptr;
    tn_status rc = TN_OK;
    cudaError_t err = cudaSuccess;
    const uint64_t mm = m ? m : 1;
    if ((err = cudaMallocAsync((void **)&du, mm * 4, st)) != cudaSuccess) goto fail;
    if ((err = cudaMallocAsync((void **)&dv, mm * 4, st)) != cudaSuccess) goto fail;
    if ((err = cudaMallocAsync((void **)&dt, mm * 8, st)) != cudaSuccess) goto fail;
    if ((err = cudaMallocAsync((void **)&S, (uint64_t)n * ld * 8, st)) != cudaSuccess) goto fail;
    if ((err = cudaMallocAsync((void **)&dout, (uint64_t)n * 4, st)) != cudaSuccess) goto fail;
    if ((err = cudaMallocAsync((void **)&dam, 4, st)) != cudaSuccess) goto fail;
    if (m) {
        if ((err = cudaMemcpyAsync(du, u, m * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) goto fail;
        if ((err = cudaMemcpyAsync(dv, v, m * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) goto fail;
        if ((err = cudaMemcpyAsync(dt, t, m * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) goto fail;
    }
    if (m == 0) {
        rc = tn_init_matrix(S, n, n, nullptr, stream);
    } else {
        tn_plan *plan = nullptr;
        rc = tn_plan_create(du, dv, dt, m, n, nullptr, opt, stream, &plan);
        if (rc == TN_OK) {
            rc = tn_plan_apply(plan, S, n, nullptr, nullptr, TN_INIT_IDENTITY, stream);
            tn_plan_destroy(plan, stream);
        }
    }
    if (rc == TN_OK) rc = tn_out_sizes(S, n, n, dout, nullptr, argmax ? dam : nullptr, stream);
    if (rc == TN_OK) {
        if ((err = cudaMemcpyAsync(out_sizes, dout, (uint64_t)n * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            goto fail;
        if (argmax && (err = cudaMemcpyAsync(argmax, dam, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) goto fail;
    }
    goto done;
fail:
    tn_internal_set_cuda_error(err);
    rc = err == cudaErrorMemoryAllocation ? TN_ENOMEM : TN_ECUDA;
done:
    if (du) cudaFreeAsync(du, st);
    if (dv) cudaFreeAsync(dv, st);
    if (dt) cudaFreeAsync(dt, st);
    if (S) cudaFreeAsync(S, st);
    if (dout) cudaFreeAsync(dout, st);
    if (dam) cudaFreeAsync(dam, st);
    err = cudaStreamSynchronize(st);
    if (rc == TN_OK && err != cudaSuccess) {
        tn_internal_set_cuda_error(err);
        rc = TN_ECUDA;
    }
    return rc;
}
