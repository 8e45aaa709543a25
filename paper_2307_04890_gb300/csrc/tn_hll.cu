// HyperLogLog sketches of the components (Section 3.3, and Section 3.4 with the
// reversed sequence; Flajolet, Fusy,
// Gandouet, Meunier 2007).
//
// Node i keeps s = 2^p one-byte registers instead of a row of n bits.  Element
// x hashes to h = one SplitMix64 step (Steele, Lea, Flood 2014) from state
// (seed XOR x); its register is the top p bits of h and its rank the position
// of the first 1 among the remaining 64 - p bits (64 - p + 1 if none).  Node i
// starts as the sketch of {i}.  An event merges sketches by register-wise
// maximum, which is the union of the sketched sets, so the same schedule and
// the same column-slab streaming kernel apply with the byte-wise maximum in
// place of OR: node i's sketch stays the sketch of its in-component (of its
// out-component when the sequence is reversed).  Estimates use the harmonic
// mean of 2^M with linear counting for small sets.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "tn_internal.cuh"

namespace tn {

__device__ inline uint64_t splitmix64_once(uint64_t state)
{
    uint64_t z = state + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// one warp per row: zero the row, then set the node's own register
__global__ void hll_init_kernel(uint8_t *R, uint32_t n, uint64_t row_bytes, uint32_t p, uint64_t seed)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t i = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        uint64_t *row = reinterpret_cast<uint64_t *>(R + i * row_bytes);
        for (uint64_t w = 2 * lane; w < row_bytes / 8; w += 64) st_row16(row + w, u64x2{0ull, 0ull});
        __syncwarp();
        if (lane == 0) {
            const uint64_t h = splitmix64_once(seed ^ i);
            const uint32_t reg = (uint32_t)(h >> (64 - p));
            const uint64_t w = h << p;
            const uint32_t rank = w ? (uint32_t)__clzll((long long)w) + 1u : 64u - p + 1u;
            R[i * row_bytes + reg] = (uint8_t)rank;
        }
        __syncwarp();
    }
}

// one warp per row: sum of 2^-M over the registers and the number of zeros
__global__ void hll_estimate_kernel(const uint8_t *R, uint32_t n, uint64_t row_bytes, uint32_t p, double alpha,
                                    double *est)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t s = 1u << p;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t i = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const uint8_t *M = R + i * row_bytes;
        double z = 0.0;
        uint32_t zeros = 0;
        for (uint32_t j = lane; j < s; j += 32) {
            const uint32_t r = M[j];
            z += ldexp(1.0, -(int)r);
            zeros += r == 0;
        }
        for (int d = 16; d > 0; d >>= 1) {
            z += __shfl_xor_sync(0xffffffffu, z, d);
            zeros += __shfl_xor_sync(0xffffffffu, zeros, d);
        }
        if (lane == 0) {
            double e = alpha * (double)s * (double)s / z;
            if (e <= 2.5 * (double)s && zeros > 0) e = (double)s * log((double)s / (double)zeros);
            est[i] = e;
        }
    }
}

static int grid_rows(uint64_t rows)
{
    const uint64_t b = (rows + 7) / 8;  // 8 warps per block
    return (int)(b < 4096 ? (b ? b : 1) : 4096);
}

}  // namespace tn

using namespace tn;

extern "C" uint64_t tn_hll_row_bytes(uint32_t p)
{
    if (p < 4 || p > 16) return 0;
    return 8 * tn_row_words(8ull << p);
}

extern "C" tn_status tn_hll_sketches(const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t m, uint32_t n,
                                     uint32_t p, uint64_t seed, uint32_t flags, uint8_t *R, void *stream)
{
    if (!R || n == 0 || n >= (1u << 30) || p < 4 || p > 16 || m >= (1ull << 30) || (m > 0 && (!u || !v || !t)) ||
        (flags & ~(TN_REVERSE | TN_DIRECTED)))
        return TN_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t row_bytes = tn_hll_row_bytes(p);
    tn_internal_keep_pool();
    tn_internal_count_launches(1);
    hll_init_kernel<<<grid_rows(n), 256, 0, st>>>(R, n, row_bytes, p, seed);
    TN_CUDA_TRY(cudaGetLastError());
    if (m == 0) return TN_OK;
    const uint32_t *eu = u, *ev = v;
    const int64_t *et = t;
    uint32_t *ru = nullptr, *rv = nullptr;
    int64_t *rt = nullptr;
    if (flags & TN_REVERSE) {
        const tn_status rr = reversed_events(u, v, t, m, (flags & TN_DIRECTED) != 0, &ru, &rv, &rt, st);
        if (rr != TN_OK) return rr;
        eu = ru;
        ev = rv;
        et = rt;
    }
    // register slabs: at least 2 words, about two CTAs per SM for wide sketches
    const uint64_t ld = row_bytes / 8;
    uint64_t sw = (ld + 2 * 152 - 1) / (2 * 152);
    sw = sw < 2 ? 2 : (sw > 16 ? 16 : (sw + 1) & ~1ull);
    tn_plan_options opt;
    memset(&opt, 0, sizeof(opt));
    opt.slab_words = (uint32_t)sw;
    opt.directed = (flags & TN_DIRECTED) ? 1u : 0u;
    tn_plan *plan = nullptr;
    tn_status rc = tn_plan_create(eu, ev, et, m, n, nullptr, &opt, stream, &plan);
    if (rc == TN_OK) {
        uint64_t *S = reinterpret_cast<uint64_t *>(R);
        const uint32_t ncols = 8u << p;
        const uint32_t *src = nullptr;
        int64_t *t_last = nullptr;
        rc = apply_jobs((const tn_plan *const *)&plan, &S, &ncols, &src, &t_last, 1, kApplyMax, st);
        if (rc == TN_OK) rc = tn_plan_status(plan, stream);
        tn_plan_destroy(plan, stream);
    }
    if (ru) cudaFreeAsync(ru, st);
    if (rv) cudaFreeAsync(rv, st);
    if (rt) cudaFreeAsync(rt, st);
    return rc;
}

extern "C" tn_status tn_hll_estimate(const uint8_t *R, uint32_t n, uint32_t p, double *est, void *stream)
{
    if (!R || !est || n == 0 || p < 4 || p > 16) return TN_EINVAL;
    const uint32_t s = 1u << p;
    const double alpha = s == 16 ? 0.673 : s == 32 ? 0.697 : s == 64 ? 0.709 : 0.7213 / (1.0 + 1.079 / (double)s);
    tn_internal_count_launches(1);
    hll_estimate_kernel<<<grid_rows(n), 256, 0, (cudaStream_t)stream>>>(R, n, tn_hll_row_bytes(p), p, alpha, est);
    TN_CUDA_TRY(cudaGetLastError());
    return TN_OK;
}
