// Error of hashed estimates against exact out-component sizes (Section 4.4:
// the estimated and exact size distributions are compared with the
// Earth-Mover distance; absolute and relative errors are reported beside it).
//
// One pass over the pairs accumulates the absolute and relative errors and two
// histograms of the values.  For integer samples of equal size the
// Wasserstein-1 distance is the area between the two empirical CDFs, i.e.
// sum over integers x of |#{est <= x} - #{exact <= x}| / count; a single CTA
// scans the histogram difference to get that sum exactly, with no sort.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "tn_internal.cuh"

namespace tn {

struct ErrAccum {
    unsigned long long sum_abs, max_abs, w1_num, max_rel_bits;
    double rel_sum;
    int32_t bad;
    int32_t pad;
};

constexpr int kErrThreads = 256;
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kErrThreads)
    error_pairs_kernel(const uint32_t *est, const uint32_t *exact, uint32_t count, uint32_t max_value,
                       uint32_t *hist_est, uint32_t *hist_exact, ErrAccum *acc)
{
    unsigned long long s = 0, mx = 0, mr = 0;
    double rs = 0.0;
    bool bad = false;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const uint32_t a = est[i], b = exact[i];
        if (a > max_value || b > max_value || b == 0) {
            bad = true;
            continue;
        }
        const unsigned long long d = a > b ? a - b : b - a;
        s += d;
        mx = d > mx ? d : mx;
        const double r = (double)d / (double)b;
        rs += r;
        // non-negative doubles order like their bit patterns
        const unsigned long long rb = (unsigned long long)__double_as_longlong(r);
        mr = rb > mr ? rb : mr;
        atomicAdd(hist_est + a, 1u);
        atomicAdd(hist_exact + b, 1u);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        const unsigned long long x = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = x > mx ? x : mx;
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, mr, o);
        mr = y > mr ? y : mr;
        rs += __shfl_xor_sync(0xffffffffu, rs, o);
    }
    bad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31u) == 0) {
        if (s) atomicAdd(&acc->sum_abs, s);
        if (mx) atomicMax(&acc->max_abs, mx);
        if (mr) atomicMax(&acc->max_rel_bits, mr);
        if (rs != 0.0) atomicAdd(&acc->rel_sum, rs);
        if (bad) atomicExch(&acc->bad, 1);
    }
}

// One CTA: w1_num = sum over x in [0, max_value] of |C(x)|, C(x) = prefix sum of
// hist_est - hist_exact up to x.  Thread t owns a contiguous chunk of x.
__global__ void __launch_bounds__(kScanThreads)
    error_w1_kernel(const uint32_t *hist_est, const uint32_t *hist_exact, uint32_t max_value, ErrAccum *acc)
{
    __shared__ long long part[kScanThreads];
    __shared__ unsigned long long tot[kScanThreads / 32];
    const uint64_t len = (uint64_t)max_value + 1;
    const uint64_t chunk = (len + kScanThreads - 1) / kScanThreads;
    const uint64_t x0 = threadIdx.x * chunk, x1 = x0 + chunk < len ? x0 + chunk : len;
    long long local = 0;
    for (uint64_t x = x0; x < x1; ++x) local += (long long)hist_est[x] - (long long)hist_exact[x];
    part[threadIdx.x] = local;
    __syncthreads();
    // inclusive Hillis-Steele scan of the chunk sums
    for (int o = 1; o < kScanThreads; o <<= 1) {
        const long long v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    long long c = threadIdx.x ? part[threadIdx.x - 1] : 0;
    unsigned long long w = 0;
    for (uint64_t x = x0; x < x1; ++x) {
        c += (long long)hist_est[x] - (long long)hist_exact[x];
        w += (unsigned long long)(c < 0 ? -c : c);
    }
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if ((threadIdx.x & 31u) == 0) tot[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < kScanThreads / 32; ++i) t += tot[i];
        acc->w1_num = t;
    }
}

}  // namespace tn

using namespace tn;

extern "C" tn_status tn_error_stats_compute(const uint32_t *est, const uint32_t *exact, uint32_t count,
                                            uint32_t max_value, tn_error_stats *out, void *stream)
{
    if (!est || !exact || !out || count == 0 || max_value == 0 || max_value >= 0xFFFFFFFFu) return TN_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t len = (uint64_t)max_value + 1;
    uint32_t *hist = nullptr;
    ErrAccum *acc = nullptr;
    ErrAccum h;
    TN_CUDA_TRY(cudaMallocAsync((void **)&hist, 2 * len * sizeof(uint32_t), st));
    TN_CUDA_TRY(cudaMallocAsync((void **)&acc, sizeof(ErrAccum), st));
    TN_CUDA_TRY(cudaMemsetAsync(hist, 0, 2 * len * sizeof(uint32_t), st));
    TN_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(ErrAccum), st));
    const unsigned blocks = (count + kErrThreads - 1) / kErrThreads < 2048 ? (count + kErrThreads - 1) / kErrThreads : 2048;
    tn_internal_count_launches(2);
    error_pairs_kernel<<<blocks, kErrThreads, 0, st>>>(est, exact, count, max_value, hist, hist + len, acc);
    error_w1_kernel<<<1, kScanThreads, 0, st>>>(hist, hist + len, max_value, acc);
    TN_CUDA_TRY(cudaGetLastError());
    TN_CUDA_TRY(cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, st));
    TN_CUDA_TRY(cudaFreeAsync(hist, st));
    TN_CUDA_TRY(cudaFreeAsync(acc, st));
    TN_CUDA_TRY(cudaStreamSynchronize(st));
    if (h.bad) return TN_ERANGE;
    double max_rel;
    memcpy(&max_rel, &h.max_rel_bits, sizeof(max_rel));
    out->count = count;
    out->sum_abs = h.sum_abs;
    out->max_abs = h.max_abs;
    out->w1_num = h.w1_num;
    out->rel_sum = h.rel_sum;
    out->max_rel = max_rel;
    out->mean_abs = (double)h.sum_abs / count;
    out->mean_rel = h.rel_sum / count;
    out->w1 = (double)h.w1_num / count;
    return TN_OK;
}
