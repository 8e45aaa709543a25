// Component sizes (Section 3.1: the out-component size of node j is the number
// of ones in column j; the in-component size of node i the number of ones in
// row i; Section 3.3: both sums have the same total n * mean size).
//
// One CTA covers 1024 consecutive columns (32 lanes x one 32-bit word each)
// and a block of rows; its 8 warps take interleaved rows.  Column counts are
// accumulated in bit-sliced vertical counters: four registers hold bits 0..3
// of 32 per-column counts, so adding a row word costs a short carry chain
// instead of 32 extractions; every 15 rows the counters are flushed into
// per-thread integer counts.  Row counts come from __popc and a warp sum.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tn_internal.cuh"

namespace tn {

constexpr int kSizeWarps = 8;
constexpr uint32_t kRowsPerBlock = 2048;

__global__ void __launch_bounds__(32 * kSizeWarps)
    column_counts_kernel(const uint32_t *S32, uint32_t n_rows, uint64_t ld32, uint32_t ncols, uint32_t *out,
                         uint32_t *in)
{
    __shared__ uint32_t part[kSizeWarps][32][33];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint64_t word = (uint64_t)blockIdx.x * 32 + lane;  // 32-bit word index inside a row
    const bool live = word < ld32;
    const uint32_t r0 = blockIdx.y * kRowsPerBlock;
    const uint32_t r1 = min(n_rows, r0 + kRowsPerBlock);

    uint32_t cnt[32];
#pragma unroll
    for (int b = 0; b < 32; ++b) cnt[b] = 0;
    uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0, pending = 0;
    for (uint32_t r = r0 + warp; r < r1; r += kSizeWarps) {
        const uint32_t x = live ? __ldcs(S32 + (uint64_t)r * ld32 + word) : 0u;
        if (in) {
            uint32_t pc = __popc(x);
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) pc += __shfl_xor_sync(0xffffffffu, pc, d);
            if (lane == 0 && pc) atomicAdd(&in[r], pc);
        }
        // add x to the 4-bit vertical counters
        uint32_t carry = c0 & x;
        c0 ^= x;
        uint32_t carry2 = c1 & carry;
        c1 ^= carry;
        uint32_t carry3 = c2 & carry2;
        c2 ^= carry2;
        c3 ^= carry3;
        if (++pending == 15) {
#pragma unroll
            for (int b = 0; b < 32; ++b)
                cnt[b] += ((c0 >> b) & 1u) + (((c1 >> b) & 1u) << 1) + (((c2 >> b) & 1u) << 2) + (((c3 >> b) & 1u) << 3);
            c0 = c1 = c2 = c3 = 0;
            pending = 0;
        }
    }
#pragma unroll
    for (int b = 0; b < 32; ++b)
        cnt[b] += ((c0 >> b) & 1u) + (((c1 >> b) & 1u) << 1) + (((c2 >> b) & 1u) << 2) + (((c3 >> b) & 1u) << 3);
#pragma unroll
    for (int b = 0; b < 32; ++b) part[warp][lane][b] = cnt[b];
    __syncthreads();
    // thread t sums column (t / 32, bit t % 32) of this block over the warps
    for (uint32_t c = threadIdx.x; c < 1024; c += blockDim.x) {
        const uint32_t l = c >> 5, b = c & 31u;
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kSizeWarps; ++w) s += part[w][l][b];
        const uint64_t col = ((uint64_t)blockIdx.x * 32 + l) * 32 + b;
        if (s && col < ncols) atomicAdd(&out[col], s);
    }
}

__global__ void argmax_kernel(const uint32_t *out, uint32_t ncols, unsigned long long *best)
{
    unsigned long long key = 0;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncols; c += gridDim.x * blockDim.x) {
        const unsigned long long k = ((unsigned long long)out[c] << 32) | (0xFFFFFFFFull - c);
        key = k > key ? k : key;
    }
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, key, d);
        key = o > key ? o : key;
    }
    if ((threadIdx.x & 31u) == 0) atomicMax(best, key);
}

__global__ void argmax_finish_kernel(const unsigned long long *best, uint32_t *argmax)
{
    *argmax = (uint32_t)(0xFFFFFFFFull - (*best & 0xFFFFFFFFull));
}

}  // namespace tn

using namespace tn;

extern "C" tn_status tn_out_sizes(const uint64_t *S, uint32_t n_rows, uint32_t ncols, uint32_t *out_sizes,
                                  uint32_t *in_sizes, uint32_t *argmax, void *stream)
{
    if (!S || !out_sizes || n_rows == 0 || ncols == 0) return TN_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t ld32 = 2 * tn_row_words(ncols);
    TN_CUDA_TRY(cudaMemsetAsync(out_sizes, 0, (size_t)ncols * sizeof(uint32_t), st));
    if (in_sizes) TN_CUDA_TRY(cudaMemsetAsync(in_sizes, 0, (size_t)n_rows * sizeof(uint32_t), st));
    dim3 grid((unsigned)((ld32 + 31) / 32), (n_rows + kRowsPerBlock - 1) / kRowsPerBlock);
    tn_internal_count_launches(1);
    column_counts_kernel<<<grid, 32 * kSizeWarps, 0, st>>>(reinterpret_cast<const uint32_t *>(S), n_rows, ld32,
                                                          ncols, out_sizes, in_sizes);
    TN_CUDA_TRY(cudaGetLastError());
    if (argmax) {
        unsigned long long *best = nullptr;
        TN_CUDA_TRY(cudaMallocAsync((void **)&best, sizeof(unsigned long long), st));
        TN_CUDA_TRY(cudaMemsetAsync(best, 0, sizeof(unsigned long long), st));
        const unsigned blocks = (unsigned)((ncols + 255) / 256 < 1024 ? (ncols + 255) / 256 : 1024);
        tn_internal_count_launches(1);
        argmax_kernel<<<blocks, 256, 0, st>>>(out_sizes, ncols, best);
        tn_internal_count_launches(1);
        argmax_finish_kernel<<<1, 1, 0, st>>>(best, argmax);
        TN_CUDA_TRY(cudaGetLastError());
        TN_CUDA_TRY(cudaFreeAsync(best, st));
    }
    return TN_OK;
}
