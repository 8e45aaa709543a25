// Component sizes (Section 3.1: the out-component size of node j is the number
// of ones in column j; the in-component size of node i the number of ones in
// row i; Section 3.3: both sums have the same total n * mean size).
//
// One CTA covers 1024 consecutive columns (32 lanes x one 32-bit word each)
// and a block of rows; its 8 warps take interleaved rows.  Column counts are
// accumulated in bit-sliced vertical counters: eight registers hold bits 0..7
// of 32 per-column counts, so adding a row word costs a carry chain instead of
// 32 extractions; every 255 rows the counters are flushed into the thread's
// 32 integer counts in shared memory (registers stay free for loads in flight).  Row counts come from __popc and a warp sum.
// Each warp loads kRowBatch rows before folding any of them in, so that
// enough loads are in flight per SM to keep HBM busy.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tn_internal.cuh"

namespace tn {

constexpr int kSizeWarps = 8;
constexpr uint32_t kRowsPerBlock = 2048;
constexpr int kRowBatch = 16;
constexpr int kCounterBits = 8;  // vertical counters hold up to 2^8 - 1

__global__ void __launch_bounds__(32 * kSizeWarps, 4)
    column_counts_kernel(const uint32_t *S32, uint32_t n_rows, uint64_t ld32, uint32_t ncols, uint32_t *out,
                         uint32_t *in)
{
    __shared__ uint32_t part[kSizeWarps][32][33];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint64_t word = (uint64_t)blockIdx.x * 32 + lane;  // 32-bit word index inside a row
    const bool live = word < ld32;
    const uint32_t r0 = blockIdx.y * kRowsPerBlock;
    const uint32_t r1 = min(n_rows, r0 + kRowsPerBlock);

    uint32_t *cnt = part[warp][lane];  // this thread's 32 column counts
#pragma unroll
    for (int b = 0; b < 32; ++b) cnt[b] = 0;
    uint32_t vc[kCounterBits];
#pragma unroll
    for (int j = 0; j < kCounterBits; ++j) vc[j] = 0;
    uint32_t pending = 0;
    // adds the vertical counters into the integer counts and clears them
    auto flush = [&]() {
#pragma unroll 4
        for (int b = 0; b < 32; ++b) {
            uint32_t v = 0;
#pragma unroll
            for (int j = 0; j < kCounterBits; ++j) v |= ((vc[j] >> b) & 1u) << j;
            cnt[b] += v;
        }
#pragma unroll
        for (int j = 0; j < kCounterBits; ++j) vc[j] = 0;
        pending = 0;
    };
    for (uint32_t rb = r0 + warp; rb < r1; rb += kRowBatch * kSizeWarps) {
        uint32_t xs[kRowBatch];
#pragma unroll
        for (int k = 0; k < kRowBatch; ++k) {
            const uint32_t r = rb + k * kSizeWarps;
            xs[k] = (live && r < r1) ? __ldcs(S32 + (uint64_t)r * ld32 + word) : 0u;
        }
#pragma unroll
        for (int k = 0; k < kRowBatch; ++k) {
            const uint32_t r = rb + k * kSizeWarps;
            if (in && r < r1) {
                uint32_t pc = __popc(xs[k]);
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) pc += __shfl_xor_sync(0xffffffffu, pc, d);
                if (lane == 0 && pc) atomicAdd(&in[r], pc);
            }
            // add the row word to the vertical counters (rows past the block add 0)
            uint32_t carry = xs[k];
#pragma unroll
            for (int j = 0; j < kCounterBits; ++j) {
                const uint32_t next = vc[j] & carry;
                vc[j] ^= carry;
                carry = next;
            }
        }
        pending += kRowBatch;
        if (pending + kRowBatch > (1u << kCounterBits) - 1u) flush();
    }
    flush();
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
