// Network hashing (Section 4.1) and fusion of the hashed out-components
// (Section 4.2).
//
// Hash family (the paper's construction is garbled; this is its reading as
// Thorup-Zhang 2-character tabulation with a derived character, which the
// paper cites): for replica j the coefficients A(i, c), i < 3, c < 4, are
// ((r1 << 32) + r2) mod p with p = 2^61 - 1 and r = successive SplitMix64
// outputs reduced modulo 2^31 - 1, the stream starting at state
// splitmix64(seed XOR j).  T_i[x] is the cubic A(i,0) x^3 + ... + A(i,3) over
// GF(p) evaluated by the MultAddMod recursion acc <- x * acc + A(i, c), and
// h(u) = (T0[u & 0xFFFF] ^ T1[u >> 16] ^ T2[(u & 0xFFFF) + (u >> 16)]) mod k.
// The coefficients are derived on the host (12 per replica); the tables are
// evaluated on the fly on the device (three cubics per node).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "tn_internal.cuh"

namespace tn {

constexpr uint64_t kP61 = (1ull << 61) - 1;

// ---------------- host: coefficient derivation ----------------
static uint64_t sm64_step(uint64_t &state)
{
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void replica_coefficients(uint64_t seed, uint32_t j, uint64_t out[12])
{
    uint64_t st = seed ^ (uint64_t)j;
    uint64_t stream = sm64_step(st);
    for (int q = 0; q < 12; ++q) {
        const uint64_t hi = sm64_step(stream) % 2147483647ull;
        const uint64_t lo = sm64_step(stream) % 2147483647ull;
        out[q] = ((hi << 32) + lo) % kP61;
    }
}

// ---------------- device: arithmetic modulo 2^61 - 1 ----------------
// (a * x + c) mod p for a, c < p and x < 2^32: the 128-bit product is folded
// with 2^61 = 1 (mod p).
__device__ inline uint64_t mul_add_p61(uint64_t a, uint64_t x, uint64_t c)
{
    const uint64_t lo = a * x;
    const uint64_t hi = __umul64hi(a, x);
    uint64_t r = (lo & kP61) + ((lo >> 61) | (hi << 3));
    r = (r >= kP61) ? r - kP61 : r;
    r += c;
    r = (r >= kP61) ? r - kP61 : r;
    return r;
}

__device__ inline uint64_t cubic_p61(const uint64_t *A, uint64_t x)
{
    uint64_t acc = A[0];
    acc = mul_add_p61(acc, x, A[1]);
    acc = mul_add_p61(acc, x, A[2]);
    acc = mul_add_p61(acc, x, A[3]);
    return acc;
}

__device__ inline uint32_t bucket_of(const uint64_t *A, uint32_t u, uint32_t k)
{
    const uint64_t x0 = u & 0xFFFFu, x1 = u >> 16;
    const uint64_t h = cubic_p61(A, x0) ^ cubic_p61(A + 4, x1) ^ cubic_p61(A + 8, x0 + x1);
    return (uint32_t)(h % k);
}

__global__ void hash_nodes_kernel(const uint64_t *coef, uint32_t R, uint32_t k, uint32_t n, uint32_t *H)
{
    const uint64_t total = (uint64_t)R * n;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t j = (uint32_t)(i / n), x = (uint32_t)(i - (uint64_t)j * n);
        H[i] = bucket_of(coef + 12ull * j, x, k);
    }
}

// super-events (h_j(u), h_j(v), t) of every replica (Section 4.1)
__global__ void proxy_events_kernel(const uint32_t *u, const uint32_t *v, uint64_t m, uint32_t n, uint32_t R,
                                    const uint32_t *H, uint32_t *pu, uint32_t *pv)
{
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t a = u[e], b = v[e];
        for (uint32_t j = 0; j < R; ++j) {
            // an endpoint outside [0, n) becomes an invalid super-node, which a
            // later plan over the super-events rejects with TN_ERANGE
            pu[(uint64_t)j * m + e] = a < n ? __ldg(H + (uint64_t)j * n + a) : 0xFFFFFFFFu;
            pv[(uint64_t)j * m + e] = b < n ? __ldg(H + (uint64_t)j * n + b) : 0xFFFFFFFFu;
        }
    }
}

// ---------------- fusion ----------------
// CTA = 8 sources.  table[j * k + b] bit s = [super-node b reached from
// h_j(x_s) in proxy j] = bit h_j(x_s) of row b of P_j.  A node w belongs to
// the estimate of source s when bit s of AND_j table[j * k + h_j(w)] is set.
constexpr int kEstSources = 8;
constexpr int kEstThreads = 256;

__global__ void check_sources_kernel(const uint32_t *src, uint32_t nsrc, uint32_t n, int32_t *bad)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nsrc; i += gridDim.x * blockDim.x)
        if (src[i] >= n) atomicExch(bad, 1);
}

__global__ void __launch_bounds__(kEstThreads)
    estimate_kernel(const uint64_t *P, uint32_t R, uint32_t k, uint64_t ldk, const uint32_t *H, uint32_t n,
                    const uint32_t *src, uint32_t nsrc, uint32_t *est, uint8_t *gtable)
{
    extern __shared__ uint8_t stable[];
    __shared__ uint32_t col[kEstSources * 64];  // h_j(x_s) for up to 64 replicas
    __shared__ uint32_t cnt[kEstSources];
    const uint32_t s0 = blockIdx.x * kEstSources;
    const uint32_t ns = min((uint32_t)kEstSources, nsrc - s0);
    uint8_t *table = gtable ? gtable + (uint64_t)blockIdx.x * R * k : stable;
    for (uint32_t q = threadIdx.x; q < kEstSources * R; q += blockDim.x) {
        const uint32_t s = q / R, j = q - s * R;
        const uint32_t x = s < ns ? (src ? src[s0 + s] : s0 + s) : 0u;
        col[s * R + j] = H[(uint64_t)j * n + x];
    }
    if (threadIdx.x < kEstSources) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (uint64_t q = threadIdx.x; q < (uint64_t)R * k; q += blockDim.x) {
        const uint32_t j = (uint32_t)(q / k), b = (uint32_t)(q - (uint64_t)j * k);
        const uint64_t *row = P + ((uint64_t)j * k + b) * ldk;
        uint32_t byte = 0;
        for (uint32_t s = 0; s < ns; ++s) {
            const uint32_t c = col[s * R + j];
            byte |= (uint32_t)((__ldg(row + (c >> 6)) >> (c & 63)) & 1ull) << s;
        }
        table[q] = (uint8_t)byte;
    }
    __syncthreads();
    uint32_t c[kEstSources];
#pragma unroll
    for (int s = 0; s < kEstSources; ++s) c[s] = 0;
    const uint32_t all = (1u << ns) - 1u;
    for (uint32_t w = blockIdx.y * blockDim.x + threadIdx.x; w < n; w += gridDim.y * blockDim.x) {
        uint32_t mask = all;
        for (uint32_t j = 0; j < R && mask; ++j) mask &= table[(uint64_t)j * k + __ldg(H + (uint64_t)j * n + w)];
#pragma unroll
        for (int s = 0; s < kEstSources; ++s) c[s] += (mask >> s) & 1u;
    }
#pragma unroll
    for (int s = 0; s < kEstSources; ++s) {
        uint32_t x = c[s];
        for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
        if ((threadIdx.x & 31u) == 0 && x) atomicAdd(&cnt[s], x);
    }
    __syncthreads();
    if (threadIdx.x < ns && cnt[threadIdx.x]) atomicAdd(&est[s0 + threadIdx.x], cnt[threadIdx.x]);
}

}  // namespace tn

using namespace tn;

extern "C" tn_status tn_hash_proxy(const uint32_t *u, const uint32_t *v, uint64_t m, uint32_t n, uint32_t k,
                                   uint32_t R, uint64_t seed, uint32_t *H, uint32_t *pu, uint32_t *pv,
                                   void *stream)
{
    if (!H || n == 0 || k == 0 || R == 0 || n >= (1u << 30) || k >= (1u << 30)) return TN_EINVAL;
    if (m > 0 && (pu || pv) && (!pu || !pv || !u || !v)) return TN_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t *hcoef = (uint64_t *)malloc(12 * sizeof(uint64_t) * R);
    if (!hcoef) return TN_ENOMEM;
    for (uint32_t j = 0; j < R; ++j) replica_coefficients(seed, j, hcoef + 12ull * j);
    uint64_t *dcoef = nullptr;
    cudaError_t err = cudaMallocAsync((void **)&dcoef, 12 * sizeof(uint64_t) * R, st);
    if (err == cudaSuccess) err = cudaMemcpyAsync(dcoef, hcoef, 12 * sizeof(uint64_t) * R, cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);  // the host copy may be freed now
    free(hcoef);
    if (err != cudaSuccess) {
        tn_internal_set_cuda_error(err);
        return err == cudaErrorMemoryAllocation ? TN_ENOMEM : TN_ECUDA;
    }
    const uint64_t total = (uint64_t)R * n;
    tn_internal_count_launches(1);
    hash_nodes_kernel<<<(unsigned)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192), 256, 0, st>>>(dcoef, R,
                                                                                                          k, n, H);
    if (m > 0 && pu) {
        tn_internal_count_launches(1);
        proxy_events_kernel<<<(unsigned)((m + 255) / 256 < 8192 ? (m + 255) / 256 : 8192), 256, 0, st>>>(
            u, v, m, n, R, H, pu, pv);
    }
    TN_CUDA_TRY(cudaGetLastError());
    TN_CUDA_TRY(cudaFreeAsync(dcoef, st));
    return TN_OK;
}

extern "C" tn_status tn_hash_estimate(const uint64_t *P, uint32_t R, uint32_t k, const uint32_t *H, uint32_t n,
                                      const uint32_t *src, uint32_t nsrc, uint32_t *est, void *stream)
{
    if (!P || !H || !est || R == 0 || R > 64 || k == 0 || n == 0 || nsrc == 0) return TN_EINVAL;
    if (!src && nsrc != n) return TN_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (src) {  // validating: source ids must be node ids
        int32_t *dbad = nullptr, hbad = 0;
        TN_CUDA_TRY(cudaMallocAsync((void **)&dbad, sizeof(int32_t), st));
        TN_CUDA_TRY(cudaMemsetAsync(dbad, 0, sizeof(int32_t), st));
        tn_internal_count_launches(1);
        check_sources_kernel<<<(nsrc + 255) / 256 < 1024 ? (nsrc + 255) / 256 : 1024, 256, 0, st>>>(src, nsrc, n, dbad);
        TN_CUDA_TRY(cudaMemcpyAsync(&hbad, dbad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        TN_CUDA_TRY(cudaFreeAsync(dbad, st));
        TN_CUDA_TRY(cudaStreamSynchronize(st));
        if (hbad) return TN_ERANGE;
    }
    const uint64_t ldk = tn_row_words(k);
    const uint64_t table_bytes = (uint64_t)R * k;
    const unsigned batches = (nsrc + kEstSources - 1) / kEstSources;
    TN_CUDA_TRY(cudaMemsetAsync(est, 0, (size_t)nsrc * sizeof(uint32_t), st));
    uint8_t *gtable = nullptr;
    size_t smem = 0;
    if (table_bytes <= 200 * 1024) {
        smem = table_bytes;
        TN_CUDA_TRY(cudaFuncSetAttribute(estimate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    } else {
        TN_CUDA_TRY(cudaMallocAsync((void **)&gtable, table_bytes * batches, st));  // one table per CTA
    }
    tn_internal_count_launches(1);
    estimate_kernel<<<dim3(batches, 1), kEstThreads, smem, st>>>(P, R, k, ldk, H, n, src, nsrc, est, gtable);
    TN_CUDA_TRY(cudaGetLastError());
    if (gtable) TN_CUDA_TRY(cudaFreeAsync(gtable, st));
    return TN_OK;
}

// ---------------- fusion without allocation ----------------
// Same kernels as tn_hash_estimate; the source-check flag and the per-CTA
// tables of the global-table path live in one fixed device array of this
// module instead of the stream-ordered allocator.  Bytes [0, 4) hold the
// flag, the tables start at byte 256.
#include <mutex>

namespace tn {
static __device__ __align__(256) uint8_t g_noalloc_scratch[TN_NOALLOC_SCRATCH_BYTES];
constexpr uint64_t kNoallocTableOffset = 256;
constexpr int kNoallocMaxDevices = 64;

// Address of the scratch on the current device, looked up once per device.
static tn_status noalloc_scratch(uint8_t **out)
{
    static std::mutex mu;
    static uint8_t *addr[kNoallocMaxDevices] = {nullptr};
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) {
        tn_internal_set_cuda_error(err);
        return TN_ECUDA;
    }
    if (dev < 0 || dev >= kNoallocMaxDevices) return TN_EINVAL;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (err != cudaSuccess) {
            tn_internal_set_cuda_error(err);
            return TN_ECUDA;
        }
        addr[dev] = (uint8_t *)p;
    }
    *out = addr[dev];
    return TN_OK;
}
}  // namespace tn

extern "C" tn_status tn_hash_estimate_noalloc(const uint64_t *P, uint32_t R, uint32_t k, const uint32_t *H,
                                              uint32_t n, const uint32_t *src, uint32_t nsrc, uint32_t *est,
                                              void *stream)
{
    if (!P || !H || !est || R == 0 || R > 64 || k == 0 || n == 0 || nsrc == 0) return TN_EINVAL;
    if (!src && nsrc != n) return TN_EINVAL;
    const uint64_t ldk = tn_row_words(k);
    const uint64_t table_bytes = (uint64_t)R * k;
    const unsigned batches = (nsrc + kEstSources - 1) / kEstSources;
    const bool smem_table = table_bytes <= 200 * 1024;
    if (!smem_table && table_bytes * batches > TN_NOALLOC_TABLE_BYTES) return TN_ESCRATCH;
    uint8_t *scratch = nullptr;
    const tn_status s = noalloc_scratch(&scratch);
    if (s != TN_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (src) {  // validating: source ids must be node ids
        int32_t *dbad = reinterpret_cast<int32_t *>(scratch), hbad = 0;
        TN_CUDA_TRY(cudaMemsetAsync(dbad, 0, sizeof(int32_t), st));
        tn_internal_count_launches(1);
        check_sources_kernel<<<(nsrc + 255) / 256 < 1024 ? (nsrc + 255) / 256 : 1024, 256, 0, st>>>(src, nsrc, n, dbad);
        TN_CUDA_TRY(cudaMemcpyAsync(&hbad, dbad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        TN_CUDA_TRY(cudaStreamSynchronize(st));
        if (hbad) return TN_ERANGE;
    }
    TN_CUDA_TRY(cudaMemsetAsync(est, 0, (size_t)nsrc * sizeof(uint32_t), st));
    size_t smem = 0;
    uint8_t *gtable = nullptr;
    if (smem_table) {
        smem = table_bytes;
        TN_CUDA_TRY(cudaFuncSetAttribute(estimate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    } else {
        gtable = scratch + kNoallocTableOffset;  // every byte is written by its CTA before it is read
    }
    tn_internal_count_launches(1);
    estimate_kernel<<<dim3(batches, 1), kEstThreads, smem, st>>>(P, R, k, ldk, H, n, src, nsrc, est, gtable);
    TN_CUDA_TRY(cudaGetLastError());
    return TN_OK;
}
