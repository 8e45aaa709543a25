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
constexpr uint32_t kBitsliceMinSources = 256;  // from here on the bit-sliced fusion is used
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

// ---------------- fusion, bit-sliced over sources ----------------
// For many sources the fusion is reorganised around a transposed table:
//   T[j][b] = bitset over the chunk's sources, bit s = bit h_j(x_s) of row b of P_j
// (Section 4.2: super-node b reaches h_j(x_s) in proxy j).  Then
//   est(x_s) = #{w : bit s of AND_j T[j][h_j(w)]},
// i.e. a column count of the n x nsrc boolean matrix whose row w is the AND
// of R rows of T -- the same vertical-counter column count as the exact
// out-sizes.  T rows are padded like component-matrix rows (tn_row_words).
constexpr int kTabThreads = 256;
constexpr uint32_t kTabRows = 64;       // proxy rows per CTA
constexpr uint32_t kTabSources = 8192;  // sources per CTA (their columns cached in shared memory)

__global__ void __launch_bounds__(kTabThreads)
    bitslice_table_kernel(const uint64_t *P, uint32_t k, uint64_t ldk, const uint32_t *H, uint32_t n,
                          const uint32_t *src, uint32_t s0, uint32_t ns, uint64_t ldT32, uint32_t *T)
{
    __shared__ uint32_t col[kTabSources];
    const uint32_t j = blockIdx.z;
    const uint32_t c0 = blockIdx.y * kTabSources;  // first source of this CTA, relative to the chunk
    const uint32_t cn = min(kTabSources, ns - c0);
    for (uint32_t q = threadIdx.x; q < cn; q += blockDim.x) {
        const uint32_t x = src ? src[s0 + c0 + q] : s0 + c0 + q;
        col[q] = H[(uint64_t)j * n + x];
    }
    __syncthreads();
    const uint32_t b0 = blockIdx.x * kTabRows;
    const uint32_t b1 = min(k, b0 + kTabRows);
    // thread t builds 32-bit words (32 sources) of each row
    const uint32_t words = (cn + 31) / 32;
    for (uint32_t b = b0; b < b1; ++b) {
        const uint64_t *row = P + ((uint64_t)j * k + b) * ldk;
        for (uint32_t wd = threadIdx.x; wd < words; wd += blockDim.x) {
            uint32_t bits = 0;
            const uint32_t base = wd * 32;
#pragma unroll 8
            for (uint32_t i = 0; i < 32; ++i) {
                const uint32_t q = base + i;
                if (q < cn) {
                    const uint32_t c = col[q];
                    bits |= (uint32_t)((__ldg(row + (c >> 6)) >> (c & 63)) & 1ull) << i;
                }
            }
            T[((uint64_t)j * k + b) * ldT32 + c0 / 32 + wd] = bits;
        }
    }
}

constexpr int kCountWarps = 8;
constexpr uint32_t kCountNodes = 4096;  // nodes w per CTA

__global__ void __launch_bounds__(32 * kCountWarps)
    bitslice_count_kernel(const uint32_t *T, uint64_t ldT32, uint32_t R, uint32_t k, const uint32_t *H, uint32_t n,
                          uint32_t ns, uint32_t *est)
{
    __shared__ uint32_t part[kCountWarps][32][33];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint64_t word = (uint64_t)blockIdx.x * 32 + lane;  // 32-bit word of a T row (32 sources)
    const bool live = word < (ns + 31) / 32;                  // words the table kernel wrote
    const uint32_t w0 = blockIdx.y * kCountNodes;
    const uint32_t w1 = min(n, w0 + kCountNodes);
    uint32_t cnt[32];
#pragma unroll
    for (int b = 0; b < 32; ++b) cnt[b] = 0;
    uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0, pending = 0;
    for (uint32_t w = w0 + warp; w < w1; w += kCountWarps) {
        uint32_t x = live ? 0xFFFFFFFFu : 0u;
        for (uint32_t j = 0; j < R && x; ++j) {
            const uint32_t b = __ldg(H + (uint64_t)j * n + w);
            x &= __ldg(T + ((uint64_t)j * k + b) * ldT32 + word);
        }
        // add x to the 4-bit vertical counters
        const uint32_t carry = c0 & x;
        c0 ^= x;
        const uint32_t carry2 = c1 & carry;
        c1 ^= carry;
        const uint32_t carry3 = c2 & carry2;
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
    for (uint32_t c = threadIdx.x; c < 1024; c += blockDim.x) {
        const uint32_t l = c >> 5, bit = c & 31u;
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kCountWarps; ++w) s += part[w][l][bit];
        const uint64_t q = ((uint64_t)blockIdx.x * 32 + l) * 32 + bit;
        if (s && q < ns) atomicAdd(&est[q], s);
    }
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

static tn_status estimate_bitsliced(const uint64_t *P, uint32_t R, uint32_t k, uint64_t ldk, const uint32_t *H,
                                    uint32_t n, const uint32_t *src, uint32_t nsrc, uint32_t *est, cudaStream_t st)
{
    // sources in chunks whose table stays within 2 GiB
    uint32_t chunk = nsrc < 65536u ? nsrc : 65536u;
    while (chunk > 1024 && (uint64_t)R * k * tn_row_words(chunk) * 8 > (2ull << 30)) chunk /= 2;
    const uint64_t ldT32 = 2 * tn_row_words(chunk);
    uint32_t *T = nullptr;
    TN_CUDA_TRY(cudaMallocAsync((void **)&T, (uint64_t)R * k * ldT32 * 4, st));
    for (uint32_t s0 = 0; s0 < nsrc; s0 += chunk) {
        const uint32_t ns = nsrc - s0 < chunk ? nsrc - s0 : chunk;
        const uint64_t ld32 = 2 * tn_row_words(ns);
        // the count kernel reads only the ceil(ns / 32) words the table kernel writes
        tn_internal_count_launches(2);
        bitslice_table_kernel<<<dim3((k + kTabRows - 1) / kTabRows, (ns + kTabSources - 1) / kTabSources, R),
                                kTabThreads, 0, st>>>(P, k, ldk, H, n, src, s0, ns, ld32, T);
        bitslice_count_kernel<<<dim3((unsigned)((ld32 + 31) / 32), (n + kCountNodes - 1) / kCountNodes),
                                32 * kCountWarps, 0, st>>>(T, ld32, R, k, H, n, ns, est + s0);
        TN_CUDA_TRY(cudaGetLastError());
    }
    TN_CUDA_TRY(cudaFreeAsync(T, st));
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
    if (nsrc >= kBitsliceMinSources) return estimate_bitsliced(P, R, k, ldk, H, n, src, nsrc, est, st);
    uint8_t *gtable = nullptr;
    size_t smem = 0;
    if (table_bytes <= 200 * 1024) {
        smem = table_bytes;
        TN_CUDA_TRY(tn_internal_allow_max_dyn_smem((const void *)estimate_kernel));
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
// For callers that cannot allocate device memory during a call (code inside
// another framework's memory budget, latency-bound loops).  Same result as
// tn_hash_estimate, but only its byte-table fusion (one CTA per 8 sources):
// the bit-sliced path for many sources needs R * k * nsrc / 8 bytes of
// transposed tables, more than a fixed array should hold, so every call here
// reads H once per 8 sources (about ceil(nsrc / 8) * R * n * 4 bytes).  The
// source-check flag and the per-CTA tables of the global-table path live in
// one fixed device array of this module instead of the stream-ordered
// allocator.  Host code never uses the array's name as an
// address: the address comes from cudaGetSymbolAddress, per device.  Bytes [0, 4) hold the
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
        TN_CUDA_TRY(tn_internal_allow_max_dyn_smem((const void *)estimate_kernel));
    } else {
        gtable = scratch + kNoallocTableOffset;  // every byte is written by its CTA before it is read
    }
    tn_internal_count_launches(1);
    estimate_kernel<<<dim3(batches, 1), kEstThreads, smem, st>>>(P, R, k, ldk, H, n, src, nsrc, est, gtable);
    TN_CUDA_TRY(cudaGetLastError());
    return TN_OK;
}
