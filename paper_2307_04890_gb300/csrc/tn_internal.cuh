// Internal helpers shared by the libtn translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tn.h"

#define TN_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t err_ = (expr);                          \
        if (err_ != cudaSuccess) {                          \
            tn_internal_set_cuda_error(err_);               \
            return err_ == cudaErrorMemoryAllocation ? TN_ENOMEM : TN_ECUDA; \
        }                                                   \
    } while (0)

void tn_internal_set_cuda_error(cudaError_t err);
// Keeps memory freed to the current device's stream-ordered pool cached for
// reuse instead of returning it to the driver at every synchronisation.
void tn_internal_keep_pool(void);
// Raises a kernel's dynamic shared-memory limit to everything the device allows
// beside the kernel's static shared memory.  Always the same value for a given
// kernel, so concurrent callers (threads, streams) cannot undo each other.
cudaError_t tn_internal_allow_max_dyn_smem(const void *kernel);
// Adds `count` to the process-wide kernel launch counter (tn_kernel_launches).
void tn_internal_count_launches(uint64_t count);
// Waits on the host for the work enqueued on `stream` so far, sleeping rather
// than spinning (an event with blocking synchronisation, one per host thread
// and device): many threads waiting at once (the serving engine's workers)
// then leave the host cores to the threads that have work.
cudaError_t tn_internal_stream_wait(cudaStream_t stream);

namespace tn {

// Bounded device-side waits: a wait that has not completed after this many
// polls (each poll suspends for up to ~1 us) records TN_ETIMEOUT and gives up.
constexpr uint32_t kWaitPolls = 1u << 22;

// Op encoding of the row-update schedule (see tn_plan.cu).
//   a: bits 31..30 = kind, bits 29..0 = destination node / temp id
//   b: EVENT / ONEWAY / COPY: source node id;  PULL: index into the aux list
// aux list of a PULL at index b: aux[b] = count c, aux[b+1 .. b+c] = source
// references (bit 31 set = temp slot, else node id).
enum OpKind : uint32_t { kEvent = 0u, kOneway = 1u, kCopy = 2u, kPull = 3u };
constexpr uint32_t kKindShift = 30;
constexpr uint32_t kIdMask = (1u << 30) - 1u;
constexpr uint32_t kTempRef = 1u << 31;
constexpr uint32_t kNoRef = 0xFFFFFFFFu;  // empty slot in a batch of source references

__host__ __device__ inline uint32_t op_a(uint32_t kind, uint32_t id) { return (kind << kKindShift) | id; }

// Work items of the streaming kernel.  The planner emits one item per window
// whose rows fit the kernel's shared-memory row buffer (a "local record") and
// one item per tile of ops for the other windows ("global tiles").  Items are
// copied whole into one shared-memory staging buffer of kStageBytes.
//   local record (uint32 words): D, T, nlev, nops | rows[D] (node ids) |
//     lvl[nlev + 1] (op offsets) | ops[nops] | aux[...] | zero padding to 16 B.
//     Rows are named by local slots: 0..D-1 the window's rows, D..D+T-1 saved
//     copies.  op = kind << 30 | la << 29 | lb << 28 | a << 14 | b  (PULL: b =
//     aux offset).  la / lb mark the op that writes row a / b for the last time
//     in the window: its result is also stored to the matrix right away, so the
//     write-back runs during the levels instead of after them, and rows that
//     are only read are never written back.
//   global tile: uint2 ops as above (node ids, absolute aux indices).
// item = {offset in 8-byte units, count (global: ops; local: 8-byte units), flags, 0}
constexpr uint32_t kStageBytes = 16384;
constexpr uint32_t kTileOps = kStageBytes / 8 - 2;
constexpr uint32_t kItemLocal = 1u;
constexpr uint32_t kItemLevelEnd = 2u;
constexpr uint32_t kLocalBits = 14;
constexpr uint32_t kLocalMask = 0x3FFFu;
constexpr uint32_t kLocalSlotLimit = 0x3FFFu;  // above the 10,240 slots a 160 KB row buffer can hold
// Widest column slab of one CTA: 128 words (1 KB row segments).
constexpr uint32_t kMaxSlabWords = 128;
constexpr uint32_t kLastA = 1u << 29;
constexpr uint32_t kLastB = 1u << 28;

__host__ __device__ inline uint32_t local_op(uint32_t kind, uint32_t a, uint32_t b)
{
    return (kind << kKindShift) | (a << kLocalBits) | b;
}

__device__ inline void record_status(int32_t *status, int32_t code)
{
    if (status) atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------------------
// mbarrier and bulk-copy (TMA, non-tensor) PTX wrappers
// ---------------------------------------------------------------------------
__device__ inline uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ inline void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ inline void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ inline void mbar_arrive(uint64_t *bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ inline void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// One poll: true once the phase with the given parity has completed.
__device__ inline bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity), "r"(1000u)
        : "memory");
    return done != 0;
}

// Bounded wait; returns false on timeout.
__device__ inline bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    for (uint32_t i = 0; i < kWaitPolls; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Bulk global -> shared copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned), completion signalled on `bar` as transaction bytes.
__device__ inline void bulk_g2s(void *smem_dst, const void *gmem_src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(smem_dst)),
        "l"(gmem_src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// 128-bit row-segment access (L2-cached, not allocated in L1)
// ---------------------------------------------------------------------------
struct u64x2 {
    uint64_t x, y;
};

__device__ inline u64x2 ld_row16(const uint64_t *p)
{
    u64x2 r;
    asm volatile("ld.global.cg.v2.u64 {%0, %1}, [%2];" : "=l"(r.x), "=l"(r.y) : "l"(p) : "memory");
    return r;
}

__device__ inline void st_row16(uint64_t *p, u64x2 r)
{
    asm volatile("st.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(r.x), "l"(r.y) : "memory");
}

__device__ inline u64x2 or16(u64x2 a, u64x2 b) { return u64x2{a.x | b.x, a.y | b.y}; }

// Combine of two row chunks: OR of bitsets (component matrix), or byte-wise
// maximum (HyperLogLog registers, one byte each).
__device__ inline uint64_t max8x8(uint64_t a, uint64_t b)
{
    const uint32_t lo = __vmaxu4((uint32_t)a, (uint32_t)b);
    const uint32_t hi = __vmaxu4((uint32_t)(a >> 32), (uint32_t)(b >> 32));
    return ((uint64_t)hi << 32) | lo;
}

template <bool kMax>
__device__ inline u64x2 combine16(u64x2 a, u64x2 b)
{
    if (kMax) return u64x2{max8x8(a.x, b.x), max8x8(a.y, b.y)};
    return or16(a, b);
}

// ---------------------------------------------------------------------------
// Block-wide exclusive scan of an array (generic pointer: shared or global).
// All threads of the block must call it; returns the total.  `warp_sums` must
// hold 32 entries of shared memory.
// ---------------------------------------------------------------------------
__device__ inline uint32_t warp_incl_scan(uint32_t x)
{
    const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= (uint32_t)d) x += y;
    }
    return x;
}

__device__ inline uint32_t block_excl_scan_value(uint32_t x, uint32_t *warp_sums, uint32_t *total)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t nwarps = (blockDim.x + 31u) >> 5;
    uint32_t incl = warp_incl_scan(x);
    if (lane == 31u) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < nwarps ? warp_sums[lane] : 0u;
        uint32_t si = warp_incl_scan(s);
        if (lane < nwarps) warp_sums[lane] = si - s;
        if (lane == nwarps - 1u) *total = si;
    }
    __syncthreads();
    uint32_t r = warp_sums[warp] + incl - x;
    __syncthreads();
    return r;
}

__device__ inline uint32_t block_excl_scan_array(uint32_t *a, uint32_t len, uint32_t *warp_sums, uint32_t *total)
{
    const uint32_t per = (len + blockDim.x - 1u) / blockDim.x;
    const uint32_t b = threadIdx.x * per;
    const uint32_t e = min(len, b + per);
    uint32_t sum = 0;
    for (uint32_t i = b; i < e; ++i) sum += a[i];
    uint32_t off = block_excl_scan_value(sum, warp_sums, total);
    for (uint32_t i = b; i < e; ++i) {
        uint32_t x = a[i];
        a[i] = off;
        off += x;
    }
    __syncthreads();
    return *total;
}

}  // namespace tn

// Plan object (opaque in the ABI).
struct tn_plan {
    int device;
    uint64_t m;
    uint32_t n;
    uint64_t windows, levels, ops, aux, temps, big_windows, local_windows, items, blob8;
    int64_t t_first, t_last;
    uint32_t slab_words;  // 64-bit words of every row owned by one CTA (the widest, with wave_ctas)
    uint32_t wave_ctas;   // 0, or the number of CTAs one matrix is spread over
    uint32_t dcap;        // row slots of the kernel's shared-memory row buffer
    uint32_t resident;    // 0, or 64-bit words of every row one CTA keeps in shared memory
    uint2 *d_blob;        // [blob8 + 2]  item payloads (8-byte units)
    uint4 *d_items;       // [items]      work items in execution order
    uint32_t *d_aux;      // [aux]        source lists of global PULL ops
    int64_t *d_tbounds;   // [2]          t_first, t_last
    int32_t *d_status;    // [1]          first asynchronous error
    int status_shared;    // d_status belongs to the owner (tn::plan_use_status), not to the plan
};

namespace tn {
// Resident-slab form (tn_plan_options.resident_words): whether a network of
// `rows` rows and `temps` saved-row slots fits one CTA's shared memory at
// `words` 64-bit words per row, beside the smallest schedule ring; and the
// largest row count that fits with no saved rows (0 for an unsupported width).
bool resident_fits(uint64_t rows, uint64_t temps, uint32_t words);
uint32_t resident_max_rows(uint32_t words);
// Internal apply flag: combine rows by byte-wise maximum (HyperLogLog
// registers) instead of OR; no initialisation.
constexpr uint32_t kApplyMax = 1u << 16;
// Launch the column-slab streaming kernel for a list of (plan, matrix) jobs.
tn_status apply_jobs(const tn_plan *const *plans, uint64_t *const *S, const uint32_t *ncols,
                     const uint32_t *const *src, int64_t *const *t_last, uint32_t count, uint32_t flags,
                     cudaStream_t stream);
// Online state in two-stream mode (used by the serving engine): its matrix
// updates (and node growth) run on `apply_stream`, while the stream given to
// each tn_online_push carries the copies and the scheduling, so scheduling a
// batch never waits for the update of the one before.  Must be called right
// after tn_online_create, with the matrix's initialisation complete on both
// streams.  Up to kOnlineFlight applied batches stay in flight; a device error
// of one is returned once that batch has finished, and always by
// tn_online_status.
constexpr uint32_t kOnlineFlight = 8;
tn_status online_use_apply_stream(tn_online *online, cudaStream_t apply_stream);
// Two-stream mode: the device status word every batch's plan records errors
// in (0 = none), for a caller that copies it out behind the updates.
const int32_t *online_status_word(const tn_online *online);
// tn_plan_create without its last host wait: the plan's device buffers are
// written by work enqueued on `stream`, so a use on another stream must first
// wait for an event recorded on `stream` after this call.
tn_status plan_create_ordered(const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t m, uint32_t n,
                              const tn_plan_options *opt, cudaStream_t stream, tn_plan **plan_out);
// Points a plan's status word at `status` (owned by the caller, e.g. one word
// for every batch of an online state, so an error gates the later batches and
// is read once); the plan's own word is released on `stream`.
tn_status plan_use_status(tn_plan *plan, int32_t *status, cudaStream_t stream);
// Reversed copy of an event sequence (Section 3.4): event m-1-e becomes event e,
// t -> ~t; with `turn` the endpoints are swapped (directed events).  The three
// arrays come from the stream-ordered allocator; the caller frees them.
tn_status reversed_events(const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t m, bool turn,
                          uint32_t **ru, uint32_t **rv, int64_t **rt, cudaStream_t st);
}  // namespace tn
