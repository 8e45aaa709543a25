// Column-slab streaming of a scheduled event batch into component matrices.
//
// Algorithm 1 (Section 3.1) updates whole rows, but bit column j of the matrix
// (the out-component of source j) evolves independently of every other column.
// Each CTA therefore owns a slab of `sw` consecutive 64-bit words of every row
// (64*sw source columns, 2 <= sw <= 128) and streams the whole level-ordered
// schedule over it:
//   * a producer warp copies the schedule, item by item, into a ring of shared
//     memory stages with bulk asynchronous copies (cp.async.bulk, completion on
//     an mbarrier), so the ops are read from L2/HBM once per CTA and without
//     occupying the consumer threads;
//   * consumer warps (12 when the CTA holds its SM alone, 4 when two CTAs share
//     an SM) apply an item: a window whose rows fit the shared-memory row
//     buffer ("local record") is gathered, updated level by level in shared
//     memory and written through at each row's last write; a tile of ops on
//     rows in HBM ("global tile") runs through a private per-thread ring of
//     cp.async copies, with hub PULLs as L2 OR-reductions.  The per-item named
//     barrier orders one level's stores before the next level's loads.
// All waits are bounded (TN_ETIMEOUT).  The per-item barrier is a reduction
// (bar.red.or) of every consumer's stop condition, so all consumers leave the
// loop at the same barrier and none can be left waiting on it.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "tn_internal.cuh"

namespace tn {

// Consumer warps per CTA, chosen at launch: 12 when a CTA's row buffer leaves
// no room for a second CTA on the SM, 4 when two CTAs share an SM (both then
// fit in the register file).  The producer is one more warp.
constexpr int kWarpsAlone = 12;
constexpr int kWarpsShared = 4;
constexpr int kMaxThreads = 32 * kWarpsAlone + 32;
constexpr int kStages = 2;
constexpr uint32_t kEndItem = 0xFFFFFFFFu;
constexpr int kMaxPlans = 24;  // networks per launch
constexpr int kMaxJobs = 2 * kMaxPlans;  // a network spread over a wave has CTAs of two widths

struct Job {
    const uint2 *blob;
    const uint4 *items;
    const uint32_t *aux;
    uint64_t nitems;
    uint64_t *S;
    uint64_t ld;    // row stride in words
    uint64_t *tmp;  // saved-row slots of global windows, ld words each
    int32_t *status;
    uint64_t w_begin;  // first row word of the job's first CTA
    uint32_t sw;    // slab words per CTA (even, 2..kMaxSlabWords)
    uint32_t cpr;   // 16-byte chunks of a row segment = sw / 2
    uint32_t cta_begin;
    uint32_t dcap;  // row slots of the shared-memory row buffer
    // resident-slab form (rw > 0): each CTA keeps rw words of every row in shared memory
    uint32_t rw;     // words of every row per CTA (1, 2 or 4), 0 = column-slab form
    uint32_t rows;   // rows of the matrix (node count of the plan)
    uint32_t ntemp;  // saved-row slots of the plan's tie groups
    uint64_t blob8;  // schedule length in 8-byte units
};

struct JobList {
    Job job[kMaxJobs];
    uint32_t count;
    uint32_t smem_bytes;  // dynamic shared memory of the launch
};

struct StageHdr {
    uint32_t count;  // ops (global tile) or 8-byte units (local record); kEndItem = stop
    uint32_t off;    // global tile: index of its first op in the stage (0 or 1)
    uint32_t local;  // 1 = local record
    uint32_t pad;
};

__device__ inline uint32_t find_job(const JobList &jl, uint32_t cta)
{
    uint32_t j = 0;
    while (j + 1 < jl.count && jl.job[j + 1].cta_begin <= cta) ++j;
    return j;
}

// A consumer thread's place in the slab: `cpr` consecutive threads share one row
// segment (one 16-byte chunk each) and `stride` row segments are handled at once.
struct Lane {
    uint32_t chunk, lane0, stride, cpr;
    uint64_t col;  // first word of this thread's chunk
    bool active;   // chunk inside the matrix and thread inside the row groups
};

// consumer threads of this launch (all warps but the producer)
__device__ inline uint32_t consumers() { return blockDim.x - 32u; }

__device__ inline Lane make_lane(const Job &J, uint32_t ct, uint64_t w0)
{
    Lane L;
    L.cpr = J.cpr;
    L.chunk = ct % L.cpr;
    L.lane0 = ct / L.cpr;
    L.stride = consumers() / L.cpr;
    L.col = w0 + 2ull * L.chunk;
    L.active = L.lane0 < L.stride && L.col < J.ld;
    return L;
}

__device__ inline uint64_t *row_ptr(const Job &J, uint32_t ref, uint64_t col)
{
    if (ref & kTempRef) return J.tmp + (uint64_t)(ref & ~kTempRef) * J.ld + col;
    return J.S + (uint64_t)ref * J.ld + col;
}

__device__ inline void consumers_sync() { asm volatile("bar.sync 1, %0;" ::"r"(consumers()) : "memory"); }
__device__ inline void consumers_sync(uint32_t count) { asm volatile("bar.sync 1, %0;" ::"r"(count) : "memory"); }

// Barrier of the consumer warps (named barrier 1) that also ORs a predicate
// across them, so that every consumer takes the same decision to stop.
__device__ inline bool consumers_sync_or(bool p, uint32_t count)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred ip, op;\n\t"
        "setp.ne.u32 ip, %1, 0;\n\t"
        "bar.red.or.pred op, 1, %2, ip;\n\t"
        "selp.u32 %0, 1, 0, op;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)p), "r"(count)
        : "memory");
    return r != 0;
}

__device__ inline bool consumers_sync_or(bool p)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred ip, op;\n\t"
        "setp.ne.u32 ip, %1, 0;\n\t"
        "bar.red.or.pred op, 1, %2, ip;\n\t"
        "selp.u32 %0, 1, 0, op;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)p), "r"(consumers())
        : "memory");
    return r != 0;
}

__device__ inline void cp_async16(void *smem_dst, const void *gmem_src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem_dst)), "l"(gmem_src) : "memory");
}

__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ inline u64x2 lds16(const u64x2 *p)
{
    u64x2 r;
    asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(r.x), "=l"(r.y) : "r"(smem_addr(p)) : "memory");
    return r;
}

__device__ inline void sts16(u64x2 *p, u64x2 v)
{
    asm volatile("st.shared.v2.u64 [%0], {%1, %2};" ::"r"(smem_addr(p)), "l"(v.x), "l"(v.y) : "memory");
}

// ---------------------------------------------------------------------------
// global tile: ops name rows by node id and read/write the matrix directly
// ---------------------------------------------------------------------------
// PULL: S[x] |= OR of the listed source rows (aux[b] = count, then refs)
template <bool kMax>
__device__ inline void apply_pull(const Job &J, uint32_t x, uint32_t b, uint64_t col)
{
    uint64_t *pd = J.S + (uint64_t)x * J.ld + col;
    u64x2 acc = ld_row16(pd);
    const uint32_t c = __ldg(J.aux + b);
    for (uint32_t i = 0; i < c; i += 8) {
        uint32_t ref[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) ref[k] = (i + k < c) ? __ldg(J.aux + b + 1 + i + k) : kNoRef;
        u64x2 r[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            r[k] = (ref[k] != kNoRef) ? ld_row16(row_ptr(J, ref[k], col)) : u64x2{0, 0};
#pragma unroll
        for (int k = 0; k < 8; ++k) acc = combine16<kMax>(acc, r[k]);
    }
    st_row16(pd, acc);
}

// Direct form, for row buffers too small to stage a chunk: four ops in flight per thread.
template <bool kMax>
__device__ inline void apply_tile_direct(const Job &J, const uint2 *ops, uint32_t count, const Lane &L)
{
    if (!L.active) return;  // partial last slab, or a thread outside the row groups
    const uint64_t col = L.col;
    const uint32_t stride = L.stride;
    for (uint32_t o = L.lane0; o < count; o += 4 * stride) {
        uint2 op[4];
        bool live[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t idx = o + k * stride;
            live[k] = idx < count;
            op[k] = live[k] ? ops[idx] : make_uint2(0u, 0u);
        }
        // loads of all four ops first (they are independent inside a level)
        u64x2 ra[4], rb[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t kind = op[k].x >> kKindShift;
            if (!live[k] || kind == kPull) continue;
            if (kind != kCopy) ra[k] = ld_row16(J.S + (uint64_t)(op[k].x & kIdMask) * J.ld + col);
            rb[k] = ld_row16(J.S + (uint64_t)op[k].y * J.ld + col);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t kind = op[k].x >> kKindShift;
            if (!live[k] || kind == kPull) continue;
            const uint64_t ia = (uint64_t)(op[k].x & kIdMask) * J.ld + col;
            if (kind == kCopy) {
                st_row16(J.tmp + ia, rb[k]);
            } else {
                const u64x2 r = combine16<kMax>(ra[k], rb[k]);
                st_row16(J.S + ia, r);
                if (kind == kEvent) st_row16(J.S + (uint64_t)op[k].y * J.ld + col, r);
            }
        }
    }
    // multi-source updates of tie groups (hub rows) in a second pass
    for (uint32_t o = L.lane0; o < count; o += stride) {
        const uint2 op = ops[o];
        if ((op.x >> kKindShift) == kPull) apply_pull<kMax>(J, op.x & kIdMask, op.y, col);
    }
}

// Ops of one level are independent.  Each consumer thread takes the ops
// lane0, lane0 + stride, ... of the tile and runs them through a private ring
// of kRing op slots in shared memory (two row chunks per op): the copies of
// the op kRing - 1 places ahead are issued (cp.async, one commit group per op)
// before the current op's rows are read back, combined and stored from
// registers.  A thread reads only the slots it filled itself, so no barrier is
// needed inside a tile; the item loop's barrier orders one level's stores
// before the next level's loads.
constexpr int kRing = 8;

__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ inline void cp_async_wait_group()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ inline void red_or16(uint64_t *p, u64x2 v)
{
    asm volatile("red.global.or.b64 [%0], %1;" ::"l"(p), "l"(v.x) : "memory");
    asm volatile("red.global.or.b64 [%0], %1;" ::"l"(p + 1), "l"(v.y) : "memory");
}

// The thread's PULLs, S[x] |= OR of the listed source rows, as a flat sequence
// of (x, source) pairs through the same private ring: a source chunk is copied
// in kRing - 1 pairs ahead, then ORed into row x by a reduction at L2
// (red.global.or), so x is never loaded and the pairs of one PULL need no
// order among themselves (OR is associative and commutative).  Rows written
// by a PULL are read by no other op of the same level.
struct PullCursor {
    uint32_t o, q, c;  // op index, next source (0-based), source count
};

__device__ inline void pull_cursor_seek(PullCursor &cur, const Job &J, const uint2 *ops, uint32_t count,
                                        uint32_t stride)
{
    while (cur.o < count && cur.q >= cur.c) {
        cur.o += stride;
        while (cur.o < count && (ops[cur.o].x >> kKindShift) != kPull) cur.o += stride;
        cur.q = 0;
        cur.c = cur.o < count ? __ldg(J.aux + ops[cur.o].y) : 0u;
    }
}

__device__ inline void apply_pulls_ring(const Job &J, const uint2 *ops, uint32_t count, u64x2 *mine, const Lane &L)
{
    const uint32_t cpr = L.cpr, stride = L.stride;
    const uint64_t col = L.col;
    PullCursor in{L.lane0, 0u, 0u};
    while (in.o < count && (ops[in.o].x >> kKindShift) != kPull) in.o += stride;
    if (in.o >= count) return;
    in.c = __ldg(J.aux + ops[in.o].y);
    pull_cursor_seek(in, J, ops, count, stride);
    PullCursor out = in;
    uint32_t issued = 0, done = 0;
    auto issue = [&]() {
        if (in.o >= count) return;
        const uint32_t ref = __ldg(J.aux + ops[in.o].y + 1 + in.q);
        const uint32_t q = L.lane0 + (issued % kRing) * stride;
        cp_async16(mine + (2 * q) * cpr, row_ptr(J, ref, col));
        ++issued;
        ++in.q;
        pull_cursor_seek(in, J, ops, count, stride);
    };
#pragma unroll 1
    for (uint32_t k = 0; k < kRing - 1; ++k) {
        issue();
        cp_async_commit();
    }
#pragma unroll 1
    while (done < issued) {
        issue();
        cp_async_commit();
        cp_async_wait_group<kRing - 1>();  // pair `done` has landed
        const uint32_t q = L.lane0 + (done % kRing) * stride;
        red_or16(J.S + (uint64_t)(ops[out.o].x & kIdMask) * J.ld + col, lds16(mine + (2 * q) * cpr));
        ++done;
        ++out.q;
        pull_cursor_seek(out, J, ops, count, stride);
    }
    cp_async_wait_group<0>();
}

template <bool kMax>
__device__ inline void apply_tile(const Job &J, const uint2 *ops, uint32_t count, u64x2 *buf, uint32_t dcap,
                                  const Lane &L)
{
    const uint32_t cpr = L.cpr, stride = L.stride;
    const uint64_t col = L.col;
    if (dcap < 2u * kRing * stride) {
        apply_tile_direct<kMax>(J, ops, count, L);
        return;
    }
    if (!L.active) return;
    u64x2 *mine = buf + L.chunk;
    const uint32_t nk = count > L.lane0 ? (count - L.lane0 + stride - 1) / stride : 0;
    // ring slot r of this thread holds its op's rows in slots 2q, 2q + 1, q = lane0 + r * stride
    auto issue = [&](uint32_t k) {
        const uint2 op = ops[L.lane0 + k * stride];
        const uint32_t kind = op.x >> kKindShift;
        const uint32_t q = L.lane0 + (k % kRing) * stride;
        if (kind != kPull) {
            if (kind != kCopy) cp_async16(mine + (2 * q) * cpr, J.S + (uint64_t)(op.x & kIdMask) * J.ld + col);
            cp_async16(mine + (2 * q + 1) * cpr, J.S + (uint64_t)op.y * J.ld + col);
        }
    };
#pragma unroll 1
    for (uint32_t k = 0; k < kRing - 1; ++k) {
        if (k < nk) issue(k);
        cp_async_commit();
    }
#pragma unroll 1
    for (uint32_t k = 0; k < nk; ++k) {
        if (k + kRing - 1 < nk) issue(k + kRing - 1);
        cp_async_commit();
        cp_async_wait_group<kRing - 1>();  // op k's copies have landed
        const uint2 op = ops[L.lane0 + k * stride];
        const uint32_t kind = op.x >> kKindShift;
        if (kind == kPull) continue;
        const uint32_t q = L.lane0 + (k % kRing) * stride;
        const uint64_t ia = (uint64_t)(op.x & kIdMask) * J.ld + col;
        const u64x2 rb = lds16(mine + (2 * q + 1) * cpr);
        if (kind == kCopy) {
            st_row16(J.tmp + ia, rb);
        } else {
            const u64x2 r = combine16<kMax>(lds16(mine + (2 * q) * cpr), rb);
            st_row16(J.S + ia, r);
            if (kind == kEvent) st_row16(J.S + (uint64_t)op.y * J.ld + col, r);
        }
    }
    cp_async_wait_group<0>();
    // multi-source updates of tie groups (hub rows) in a second pass
    if (kMax) {
        for (uint32_t o = L.lane0; o < count; o += stride) {
            const uint2 op = ops[o];
            if ((op.x >> kKindShift) == kPull) apply_pull<kMax>(J, op.x & kIdMask, op.y, col);
        }
    } else {
        apply_pulls_ring(J, ops, count, mine, L);
    }
}

// ---------------------------------------------------------------------------
// local record: the window's rows are gathered into shared memory, its levels
// are applied there, and every written row goes back to the matrix from the op
// that writes it for the last time (rows that are only read are not stored)
// ---------------------------------------------------------------------------
template <bool kMax>
__device__ inline void apply_record(const Job &J, const uint32_t *rec, u64x2 *buf, const Lane &L)
{
    const uint32_t D = rec[0], nlev = rec[2], nops = rec[3];
    const uint32_t *rows = rec + 4, *lvl = rows + D, *ops = lvl + nlev + 1, *aux = ops + nops;
    const uint32_t cpr = L.cpr, lane0 = L.lane0, stride = L.stride;
    const uint64_t col = L.col;
    const bool active = L.active;
    u64x2 *mine = buf + L.chunk;  // slot q of this chunk lives at buf[q * cpr + chunk]

    if (active) {
        uint32_t d = lane0;
        for (; d + 3 * stride < D; d += 4 * stride) {
            uint32_t r[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) r[k] = rows[d + k * stride];
#pragma unroll
            for (int k = 0; k < 4; ++k) cp_async16(mine + (d + k * stride) * cpr, J.S + (uint64_t)r[k] * J.ld + col);
        }
        for (; d < D; d += stride) cp_async16(mine + d * cpr, J.S + (uint64_t)rows[d] * J.ld + col);
    }
    cp_async_wait_all();
    consumers_sync();
    for (uint32_t l = 0; l < nlev; ++l) {
        if (active) {
            const uint32_t e = lvl[l + 1];
            // two ops per step: the ops of one level touch distinct rows, so
            // both ops' loads can be issued before either op's stores
            for (uint32_t o = lvl[l] + lane0; o < e; o += 2 * stride) {
                uint32_t op[2];
                bool live[2];
                u64x2 x[2], y[2];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const uint32_t idx = o + k * stride;
                    live[k] = idx < e;
                    op[k] = live[k] ? ops[idx] : (kPull << kKindShift);
                    const uint32_t kind = op[k] >> kKindShift, a = (op[k] >> kLocalBits) & kLocalMask,
                                   b = op[k] & kLocalMask;
                    if (kind != kPull) {
                        x[k] = lds16(mine + a * cpr);
                        y[k] = lds16(mine + b * cpr);
                    }
                }
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const uint32_t kind = op[k] >> kKindShift, a = (op[k] >> kLocalBits) & kLocalMask,
                                   b = op[k] & kLocalMask;
                    // a row's last write in the window also goes to the matrix (write-through)
                    if (kind == kEvent) {
                        const u64x2 r = combine16<kMax>(x[k], y[k]);
                        sts16(mine + a * cpr, r);
                        sts16(mine + b * cpr, r);
                        if (op[k] & kLastA) st_row16(J.S + (uint64_t)rows[a] * J.ld + col, r);
                        if (op[k] & kLastB) st_row16(J.S + (uint64_t)rows[b] * J.ld + col, r);
                    } else if (kind == kOneway) {
                        const u64x2 r = combine16<kMax>(x[k], y[k]);
                        sts16(mine + a * cpr, r);
                        if (op[k] & kLastA) st_row16(J.S + (uint64_t)rows[a] * J.ld + col, r);
                    } else if (kind == kCopy) {
                        sts16(mine + a * cpr, y[k]);
                    } else if (live[k]) {
                        u64x2 acc = lds16(mine + a * cpr);
                        const uint32_t c = aux[b];
                        for (uint32_t q = 1; q <= c; ++q) acc = combine16<kMax>(acc, lds16(mine + aux[b + q] * cpr));
                        sts16(mine + a * cpr, acc);
                        if (op[k] & kLastA) st_row16(J.S + (uint64_t)rows[a] * J.ld + col, acc);
                    }
                }
            }
        }
        consumers_sync();
    }
    // no write-back pass: every written row was stored at its last write
}

// ---------------------------------------------------------------------------
// resident slab: for a network small enough that rw words of EVERY row fit in
// shared memory, the CTA loads its slab of the matrix once, applies the whole
// schedule there and stores it once; only the schedule streams from L2/HBM.
// The plan holds global tiles only (node-id ops, one level per tile or more;
// windows of a resident plan are never local records with ops).  The producer
// warp copies the schedule blob in fixed chunks of kStageBytes into a ring of
// `nst` stages with cp.async.bulk; consumers walk the item list, wait for the
// chunks an item covers, apply its ops (independent inside a level) and meet
// at a named barrier only where a level ends.  A consumer warp releases a
// chunk (one arrival on its `empty` barrier) once it has started an item past
// it, so a stage is refilled only when every warp is done with it.
// Shared memory: barriers | rows[rows] | saved rows[ntemp] | ring.
// ---------------------------------------------------------------------------
constexpr uint32_t kChunk8 = kStageBytes / 8;  // 8-byte units per ring stage
constexpr uint32_t kResidentMaxStages = 8;
constexpr uint32_t kResidentHead = 2 * kResidentMaxStages * sizeof(uint64_t);  // the ring's barriers
constexpr uint32_t kResidentMinStages = 2;
constexpr uint32_t kResidentConsumers = 256;  // consumer threads of a resident CTA (the rest exit)

template <int RW>
struct alignas(RW == 1 ? 8 : 16) RRow {
    uint64_t w[RW];
};

__host__ __device__ inline uint64_t resident_rows_bytes(uint64_t rows, uint64_t temps, uint32_t rw)
{
    return ((rows + temps) * 8ull * rw + 127ull) & ~127ull;
}

template <bool kMax, int RW>
__device__ inline RRow<RW> rcombine(RRow<RW> a, const RRow<RW> &b)
{
#pragma unroll
    for (int k = 0; k < RW; ++k) a.w[k] = kMax ? max8x8(a.w[k], b.w[k]) : (a.w[k] | b.w[k]);
    return a;
}

template <int RW>
__device__ inline RRow<RW> ld_rrow(const uint64_t *p)
{
    RRow<RW> r;
    if (RW == 1) {
        asm volatile("ld.global.cg.u64 %0, [%1];" : "=l"(r.w[0]) : "l"(p) : "memory");
    } else {
#pragma unroll
        for (int k = 0; k < RW; k += 2) {
            const u64x2 x = ld_row16(p + k);
            r.w[k] = x.x;
            r.w[k + 1] = x.y;
        }
    }
    return r;
}

template <int RW>
__device__ inline void st_rrow(uint64_t *p, const RRow<RW> &r)
{
    if (RW == 1) {
        asm volatile("st.global.u64 [%0], %1;" ::"l"(p), "l"(r.w[0]) : "memory");
    } else {
#pragma unroll
        for (int k = 0; k < RW; k += 2) st_row16(p + k, u64x2{r.w[k], r.w[k + 1]});
    }
}

// Rows of the resident slab by 32-bit shared-memory address.
template <int RW>
__device__ inline RRow<RW> lds_rrow(uint32_t a)
{
    RRow<RW> r;
    if (RW == 1) {
        asm volatile("ld.shared.u64 %0, [%1];" : "=l"(r.w[0]) : "r"(a) : "memory");
    } else {
#pragma unroll
        for (int k = 0; k < RW; k += 2)
            asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(r.w[k]), "=l"(r.w[k + 1]) : "r"(a + 8u * k) : "memory");
    }
    return r;
}

template <int RW>
__device__ inline void sts_rrow(uint32_t a, const RRow<RW> &r)
{
    if (RW == 1) {
        asm volatile("st.shared.u64 [%0], %1;" ::"r"(a), "l"(r.w[0]) : "memory");
    } else {
#pragma unroll
        for (int k = 0; k < RW; k += 2)
            asm volatile("st.shared.v2.u64 [%0], {%1, %2};" ::"r"(a + 8u * k), "l"(r.w[k]), "l"(r.w[k + 1]) : "memory");
    }
}

__device__ inline uint2 lds_op(uint32_t a)
{
    uint2 r;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "r"(a) : "memory");
    return r;
}

// One op of a global tile on the resident rows (shared address rb, node ids)
// and the saved rows (shared address tb, temp ids).
template <bool kMax, int RW>
__device__ inline void resident_op(uint2 op, uint32_t rb, uint32_t tb, const uint32_t *aux)
{
    constexpr uint32_t kRowB = 8u * RW;
    const uint32_t kind = op.x >> kKindShift, a = op.x & kIdMask;
    const uint32_t pa = rb + a * kRowB;
    if (kind == kEvent) {
        const uint32_t pb = rb + op.y * kRowB;
        const RRow<RW> r = rcombine<kMax, RW>(lds_rrow<RW>(pa), lds_rrow<RW>(pb));
        sts_rrow<RW>(pa, r);
        sts_rrow<RW>(pb, r);
    } else if (kind == kOneway) {
        sts_rrow<RW>(pa, rcombine<kMax, RW>(lds_rrow<RW>(pa), lds_rrow<RW>(rb + op.y * kRowB)));
    } else if (kind == kCopy) {
        sts_rrow<RW>(tb + a * kRowB, lds_rrow<RW>(rb + op.y * kRowB));
    } else {
        RRow<RW> acc = lds_rrow<RW>(pa);
        const uint32_t c = __ldg(aux + op.y);
        for (uint32_t q = 1; q <= c; ++q) {
            const uint32_t ref = __ldg(aux + op.y + q);
            acc = rcombine<kMax, RW>(acc, lds_rrow<RW>((ref & kTempRef) ? tb + (ref & ~kTempRef) * kRowB
                                                                     : rb + ref * kRowB));
        }
        sts_rrow<RW>(pa, acc);
    }
}

// Lane L of a warp holds item i0 + L of a batch of 32 as (offset, count |
// flags << 16); the next batch is loaded one batch ahead, so its L2 latency is
// hidden behind 32 items of work.
__device__ inline void load_item(const uint4 *items, uint32_t nitems, uint32_t i, uint32_t &off, uint32_t &cf)
{
    off = 0;
    cf = 0;
    if (i < nitems) {
        const uint4 it = __ldg(items + i);
        off = it.x;
        cf = it.y | (it.z << 16);  // count < 2^16 (at most one stage), flags < 4
    }
}

template <bool kMax, int RW>
__device__ void resident_slab(const Job &J, uint32_t smem_bytes, uint8_t *smem, uint32_t cta)
{
    __shared__ int32_t r_gate;
    using Row = RRow<RW>;
    // the job's fields in registers (the barriers' memory clobbers would reload them)
    const uint4 *const items = J.items;
    const uint32_t nitems = (uint32_t)J.nitems;
    const uint32_t *const aux = J.aux;
    const uint2 *const blob = J.blob;
    const uint64_t blob8 = J.blob8;
    int32_t *const status = J.status;
    uint64_t *const S = J.S;
    const uint64_t ld = J.ld;
    const uint32_t rows = J.rows;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + kResidentMaxStages;
    Row *R = reinterpret_cast<Row *>(smem + kResidentHead);
    const uint32_t rb = smem_addr(R), tb = rb + rows * 8u * RW;  // rows, then saved rows
    const uint32_t ring_off = kResidentHead + (uint32_t)resident_rows_bytes(rows, J.ntemp, RW);
    uint8_t *ring = smem + ring_off;
    // a power of two of stages (at least kResidentMinStages by the plan's check)
    const uint32_t fit = (smem_bytes - ring_off) / kStageBytes;
    uint32_t nst = kResidentMaxStages;
    while (nst > fit) nst >>= 1;
    const uint32_t smask = nst - 1, sshift = __ffs(nst) - 1;
    const uint64_t w0 = J.w_begin + (uint64_t)cta * RW;
    // Every chunk of the blob holds part of some item: windows' regions and
    // records are whole 16-byte units, so a window's padding unit (after an odd
    // number of ops) sits at an odd offset and never begins a chunk.  Every
    // chunk the producer copies is therefore waited for and released.
    const uint32_t nchunks = (uint32_t)((blob8 + kChunk8 - 1) / kChunk8);
    const uint32_t C = consumers() < kResidentConsumers ? consumers() : kResidentConsumers;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    if (threadIdx.x == 0) {
        r_gate = *(volatile int32_t *)status;  // an earlier error gates this job
        for (uint32_t s = 0; s < nst; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], C / 32u);
        }
        fence_mbar_init();
    }
    __syncthreads();
    if (r_gate != 0 || nitems == 0) return;  // no ops: the slab is unchanged

    if (warp == 0) {
        // ---------------- producer: the blob in fixed chunks ----------------
        if (lane == 0) {
            uint32_t c = 0;
            for (; c < nchunks; ++c) {
                const uint32_t s = c & smask;
                if (c >= nst && !mbar_wait_bounded(&empty[s], ((c >> sshift) - 1u) & 1u)) {
                    record_status(status, TN_ETIMEOUT);
                    break;
                }
                const uint64_t b8 = (uint64_t)c * kChunk8;
                uint32_t n8 = blob8 - b8 < kChunk8 ? (uint32_t)(blob8 - b8) : kChunk8;
                n8 = (n8 + 1u) & ~1u;  // whole 16-byte units (the blob has two spare units)
                mbar_arrive_expect_tx(&full[s], n8 * 8u);
                bulk_g2s(ring + (size_t)s * kStageBytes, blob + b8, n8 * 8u, &full[s]);
            }
            // no bulk copy may still be writing this CTA's shared memory at exit
            for (uint32_t q = c > nst ? c - nst : 0; q < c; ++q)
                mbar_wait_bounded(&full[q & smask], (q >> sshift) & 1u);
        }
        return;
    }
    // ---------------- consumers ----------------
    const uint32_t ct = threadIdx.x - 32;
    if (ct >= C) return;  // small levels keep few warps busy: the others leave
    {
        uint32_t i = ct;
        for (; i + 3 * C < rows; i += 4 * C) {
            Row r[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) r[k] = ld_rrow<RW>(S + (uint64_t)(i + k * C) * ld + w0);
#pragma unroll
            for (int k = 0; k < 4; ++k) R[i + k * C] = r[k];
        }
        for (; i < rows; i += C) R[i] = ld_rrow<RW>(S + (uint64_t)i * ld + w0);
    }
    // op o of the blob, from the stage of its chunk (which has landed)
    const uint32_t ringa = smem_addr(ring);
    auto op_at = [&](uint32_t o) -> uint2 {
        return lds_op(ringa + ((o / kChunk8) & smask) * kStageBytes + (o % kChunk8) * 8u);
    };
    bool failed = false;
    uint32_t waited = 0;    // chunks [0, waited) have landed, as seen by this thread
    uint32_t released = 0;  // chunks this warp has released
    uint32_t boff, bcf, noff, ncf;  // this lane's item of the current and of the next batch
    load_item(items, nitems, lane, boff, bcf);
    load_item(items, nitems, 32 + lane, noff, ncf);
    uint32_t off8 = 0, cf = 0;
    uint2 op0 = make_uint2(0u, 0u);  // this thread's first op of the next item
    bool have = false;
    // Prepares item i: releases the chunks before it, waits for the chunks it
    // covers, and fetches this thread's first op of it.
    auto prepare = [&](uint32_t i) {
        const uint32_t k = i & 31u;
        if (k == 0 && i > 0) {
            boff = noff;
            bcf = ncf;
            load_item(items, nitems, i + 32 + lane, noff, ncf);
        }
        off8 = __shfl_sync(0xffffffffu, boff, k);
        cf = __shfl_sync(0xffffffffu, bcf, k);
        const uint32_t count = cf & 0xFFFFu;
        const uint32_t c0 = off8 / kChunk8, c1 = (off8 + count - 1u) / kChunk8;
        if (released < c0 || waited <= c1) {  // a chunk boundary (one test in the common case)
            if (released < c0) {  // every lane of the warp is done with these chunks
                __syncwarp();
                if (lane == 0)
                    for (uint32_t q = released; q < c0; ++q) mbar_arrive(&empty[q & smask]);
                released = c0;
            }
            while (waited <= c1 && !failed) {
                if (mbar_wait_bounded(&full[waited & smask], (waited >> sshift) & 1u)) {
                    ++waited;
                } else {
                    record_status(status, TN_ETIMEOUT);
                    failed = true;
                }
            }
        }
        have = !failed && ct < count && !((cf >> 16) & kItemLocal);
        op0 = op_at(off8 + ct);  // always inside the ring; used only if `have`
    };
    consumers_sync(C);
    prepare(0);
    uint32_t lev = 0;
    for (uint32_t i = 0;;) {
        const uint32_t count = cf & 0xFFFFu, flags = cf >> 16, base8 = off8;
        if (have) {
            resident_op<kMax, RW>(op0, rb, tb, aux);
            for (uint32_t q = ct + C; q < count; q += C) resident_op<kMax, RW>(op_at(base8 + q), rb, tb, aux);
        }
        if (++i == nitems) break;
        prepare(i);  // item info and first op of the next item load before the barrier
        // the next level reads what this one wrote; every 64th level end also
        // agrees on stopping (a thread that gave up skips its work until then)
        if (flags & kItemLevelEnd) {
            if ((++lev & 63u) == 0) {
                if (consumers_sync_or(failed, C)) break;
            } else {
                consumers_sync(C);
            }
        }
    }
    if (consumers_sync_or(failed, C)) return;
    for (uint32_t i = ct; i < rows; i += C) st_rrow<RW>(S + (uint64_t)i * ld + w0, R[i]);
}

template <bool kMax>
__global__ void __launch_bounds__(kMaxThreads) stream_kernel(const __grid_constant__ JobList jl)
{
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t *stage = smem;  // kStages x kStageBytes
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)kStages * kStageBytes);
    uint64_t *empty = full + kStages;
    StageHdr *hdr = reinterpret_cast<StageHdr *>(empty + kStages);
    u64x2 *rowbuf = reinterpret_cast<u64x2 *>(hdr + kStages);  // 16-byte aligned
    __shared__ uint32_t producer_abort;
    __shared__ int32_t gate;

    const Job &J = jl.job[find_job(jl, blockIdx.x)];
    if (J.rw) {
        const uint32_t cta = blockIdx.x - J.cta_begin;
        if (J.rw == 1) resident_slab<kMax, 1>(J, jl.smem_bytes, smem, cta);
        else resident_slab<kMax, 2>(J, jl.smem_bytes, smem, cta);
        return;
    }
    const uint64_t w0 = J.w_begin + (uint64_t)(blockIdx.x - J.cta_begin) * J.sw;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    if (threadIdx.x == 0) {
        gate = *(volatile int32_t *)J.status;  // an earlier error gates this job
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], consumers() / 32u);
        }
        producer_abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (gate != 0) return;

    if (warp == 0) {
        // ---------------- producer: one bulk copy per item ----------------
        uint64_t slot = 0;  // stage uses so far
        int ok = 1;
        for (uint64_t i0 = 0; i0 < J.nitems && ok; i0 += 32) {
            const uint4 mine = (i0 + lane < J.nitems) ? __ldg(J.items + i0 + lane) : make_uint4(0u, 0u, 0u, 0u);
            const uint32_t nb = (J.nitems - i0 < 32) ? (uint32_t)(J.nitems - i0) : 32u;
            for (uint32_t k = 0; k < nb && ok; ++k) {
                const uint32_t off8 = __shfl_sync(0xffffffffu, mine.x, k);
                const uint32_t count = __shfl_sync(0xffffffffu, mine.y, k);
                const uint32_t flags = __shfl_sync(0xffffffffu, mine.z, k);
                const int s = (int)(slot % kStages);
                if (lane == 0) {
                    if (slot >= kStages && !mbar_wait_bounded(&empty[s], (uint32_t)((slot / kStages) - 1) & 1u)) {
                        record_status(J.status, TN_ETIMEOUT);
                        producer_abort = 1;
                        ok = 0;
                    } else {
                        uint32_t a0 = off8, n8 = count, off = 0;
                        if (!(flags & kItemLocal)) {  // global tile: start on a 16-byte boundary
                            a0 = off8 & ~1u;
                            off = off8 - a0;
                            n8 = (count + off + 1u) & ~1u;
                        }
                        hdr[s].count = count;
                        hdr[s].off = off;
                        hdr[s].local = flags & kItemLocal;
                        mbar_arrive_expect_tx(&full[s], n8 * 8u);
                        bulk_g2s(stage + (size_t)s * kStageBytes, J.blob + a0, n8 * 8u, &full[s]);
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (ok) ++slot;
            }
        }
        if (lane == 0) {
            if (ok) {
                const int s = (int)(slot % kStages);
                if (slot >= kStages && !mbar_wait_bounded(&empty[s], (uint32_t)((slot / kStages) - 1) & 1u)) {
                    record_status(J.status, TN_ETIMEOUT);
                    producer_abort = 1;
                } else {
                    hdr[s].count = kEndItem;
                    hdr[s].off = 0;
                    hdr[s].local = 0;
                    mbar_arrive(&full[s]);
                    ++slot;
                }
            }
            // no bulk copy may still be writing this CTA's shared memory at exit
            const uint64_t first = slot > (uint64_t)kStages ? slot - kStages : 0;
            for (uint64_t q = first; q < slot; ++q)
                mbar_wait_bounded(&full[q % kStages], (uint32_t)(q / kStages) & 1u);
        }
    } else {
        // ---------------- consumers ----------------
        const uint32_t ct = threadIdx.x - 32;
        const Lane L = make_lane(J, ct, w0);
        for (uint64_t it = 0;; ++it) {
            const int s = (int)(it % kStages);
            const uint32_t par = (uint32_t)(it / kStages) & 1u;
            const bool ready = mbar_wait_bounded(&full[s], par);
            if (!ready && ct == 0) record_status(J.status, TN_ETIMEOUT);
            const bool stop = !ready || *(volatile uint32_t *)&producer_abort != 0 ||
                              (ready && hdr[s].count == kEndItem);
            // level barrier: the previous item's stores are ordered before this
            // item's loads, and all consumers agree on stopping
            if (consumers_sync_or(stop)) break;
            if (hdr[s].local) {
                apply_record<kMax>(J, reinterpret_cast<const uint32_t *>(stage + (size_t)s * kStageBytes), rowbuf, L);
            } else {
                apply_tile<kMax>(J, reinterpret_cast<const uint2 *>(stage + (size_t)s * kStageBytes) + hdr[s].off,
                           hdr[s].count, rowbuf, J.dcap, L);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
    }
}

// Self-test of the bounded waits: one thread waits on an mbarrier that nothing
// ever completes, through the same bounded wait the streaming kernel uses, and
// records TN_ETIMEOUT when the wait gives up.
__global__ void wait_selftest_kernel(int32_t *status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_mbar_init();
    if (!mbar_wait_bounded(&bar, 0)) record_status(status, TN_ETIMEOUT);
}

// S <- identity (full matrix) -- Algorithm 1, first line; one row per warp step
__global__ void init_identity_kernel(uint64_t *S, uint32_t n_rows, uint64_t ld, const int32_t *status)
{
    if (*(volatile const int32_t *)status != 0) return;
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t r = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < n_rows; r += warps) {
        uint64_t *row = S + r * ld;
        const uint64_t diag = r >> 6;
        for (uint64_t w = 2 * lane; w < ld; w += 64) {
            u64x2 z{w == diag ? (1ull << (r & 63)) : 0ull, w + 1 == diag ? (1ull << (r & 63)) : 0ull};
            st_row16(row + w, z);
        }
    }
}

__global__ void zero_kernel(uint64_t *S, uint64_t total, const int32_t *status)
{
    if (*(volatile const int32_t *)status != 0) return;
    for (uint64_t i = 2 * (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x); i < total;
         i += 2 * (uint64_t)gridDim.x * blockDim.x)
        st_row16(S + i, u64x2{0ull, 0ull});
}

// column c of the matrix starts as the single source src[c]; ids >= n_rows
// are skipped and reported as TN_ERANGE
__global__ void init_sources_kernel(uint64_t *S, uint64_t ld, const uint32_t *src, uint32_t nsrc, uint32_t n_rows,
                                    int32_t *status)
{
    if (*(volatile const int32_t *)status != 0) return;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nsrc; c += gridDim.x * blockDim.x) {
        const uint32_t x = src[c];
        if (x >= n_rows) {
            record_status(status, TN_ERANGE);
            continue;
        }
        atomicOr((unsigned long long *)(S + (uint64_t)x * ld + (c >> 6)), 1ull << (c & 63));
    }
}

__global__ void check_ids_kernel(const uint32_t *ids, uint32_t count, uint32_t n, int32_t *status)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        if (ids[i] >= n) record_status(status, TN_ERANGE);
}

// Validating check that every source id is a node id (< n).
static tn_status validate_sources(const uint32_t *src, uint32_t nsrc, uint32_t n, cudaStream_t st)
{
    int32_t *d = nullptr, h = 0;
    TN_CUDA_TRY(cudaMallocAsync((void **)&d, sizeof(int32_t), st));
    TN_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(int32_t), st));
    tn_internal_count_launches(1);
    check_ids_kernel<<<(nsrc + 255) / 256 < 1024 ? (nsrc + 255) / 256 : 1024, 256, 0, st>>>(src, nsrc, n, d);
    TN_CUDA_TRY(cudaGetLastError());
    TN_CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    TN_CUDA_TRY(cudaFreeAsync(d, st));
    TN_CUDA_TRY(cudaStreamSynchronize(st));
    return (tn_status)h;
}

// batch order check (streaming, Section 3.5): the batch must start after t_last
__global__ void order_gate_kernel(const int64_t *tb, const int64_t *t_last, int32_t *status)
{
    if (*t_last >= tb[0]) record_status(status, TN_EORDER);
}

__global__ void set_t_last_kernel(const int64_t *tb, int64_t *t_last, const int32_t *status)
{
    if (*(volatile const int32_t *)status == 0) *t_last = tb[1];
}

// Column slabs of one matrix of `ld` row words: ceil(ld / sw) CTAs of sw
// words, or -- with wave > 0 -- exactly max(wave, ceil(ld / sw)) CTAs of two
// widths that differ by one unit (16 words when sw is a multiple of 16 and the
// row holds that many units, else 2 words): the wider ones first.
struct SlabSplit {
    uint64_t w_begin;
    uint32_t sw, ctas;
};

static int split_slabs(uint64_t ld, uint32_t sw, uint32_t wave, SlabSplit out[2])
{
    const uint64_t plain = (ld + sw - 1) / sw;
    if (wave == 0 || ld == 0) {
        out[0] = SlabSplit{0, sw, (uint32_t)plain};
        return 1;
    }
    const uint64_t C = wave > plain ? wave : plain;
    const uint32_t unit = (sw % 16 == 0 && ld / 16 >= C) ? 16u : 2u;
    const uint64_t units = ld / unit;  // ld is a multiple of 16
    if (units <= C) {  // no more CTAs than units: one unit each
        out[0] = SlabSplit{0, unit, (uint32_t)units};
        return 1;
    }
    const uint64_t q = units / C, r = units % C;
    int k = 0;
    if (r) out[k++] = SlabSplit{0, (uint32_t)((q + 1) * unit), (uint32_t)r};
    out[k++] = SlabSplit{r * (q + 1) * unit, (uint32_t)(q * unit), (uint32_t)(C - r)};
    return k;
}

// Dynamic shared memory the streaming kernel can use on the current device
// (the opt-in maximum minus its static shared memory), cached per device.
static uint32_t stream_smem_limit()
{
    static std::mutex mu;
    static uint32_t cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    std::lock_guard<std::mutex> lock(mu);
    if (!cached[dev]) {
        int optin = 0;
        cudaFuncAttributes fa;
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, (const void *)stream_kernel<false>) != cudaSuccess)
            return 0;
        cached[dev] = (uint32_t)(optin - (int)fa.sharedSizeBytes);
    }
    return cached[dev];
}

static int multiprocessors()
{
    static std::mutex mu;
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    std::lock_guard<std::mutex> lock(mu);
    if (!cached[dev] && cudaDeviceGetAttribute(&cached[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        cached[dev] = 0;
    return cached[dev] > 0 ? cached[dev] : 1;
}

// dynamic shared memory of a CTA that leaves room for a second one on its SM
constexpr uint64_t kHalfSmSmem = 112 * 1024;

bool resident_fits(uint64_t rows, uint64_t temps, uint32_t words)
{
    if (words != 1 && words != 2) return false;
    return kResidentHead + resident_rows_bytes(rows, temps, words) + (uint64_t)kResidentMinStages * kStageBytes <=
           stream_smem_limit();
}

uint32_t resident_max_rows(uint32_t words)
{
    if (words != 1 && words != 2) return 0;
    const uint64_t lim = stream_smem_limit();
    const uint64_t fixed = kResidentHead + (uint64_t)kResidentMinStages * kStageBytes;
    if (lim <= fixed) return 0;
    return (uint32_t)(((lim - fixed) & ~127ull) / (8ull * words));
}

static int grid_for(uint64_t work)
{
    uint64_t g = (work + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 8192 ? 8192 : g));
}


tn_status apply_jobs(const tn_plan *const *plans, uint64_t *const *S, const uint32_t *ncols,
                     const uint32_t *const *src, int64_t *const *t_last, uint32_t count, uint32_t flags,
                     cudaStream_t st)
{
    // host-side argument checks
    for (uint32_t i = 0; i < count; ++i) {
        const tn_plan *p = plans[i];
        if (!p || !S[i] || ncols[i] == 0) return TN_EINVAL;
        // the identity initialisation needs one column per node
        if ((flags & TN_INIT_IDENTITY) && !src[i] && ncols[i] != p->n) return TN_EINVAL;
    }
    const size_t smem_base = (size_t)kStages * kStageBytes + 2 * kStages * sizeof(uint64_t) + kStages * sizeof(StageHdr);
    const size_t smem_limit = stream_smem_limit();
    if ((flags & kApplyMax) || !smem_limit)
        for (uint32_t i = 0; i < count; ++i)
            if (plans[i]->resident) return TN_EINVAL;
    uint64_t *tmps[kMaxPlans];
    for (uint32_t base = 0; base < count; base += kMaxPlans) {
        const uint32_t nj = count - base < (uint32_t)kMaxPlans ? count - base : (uint32_t)kMaxPlans;
        JobList jl;
        memset(&jl, 0, sizeof(jl));
        jl.count = 0;
        uint32_t ctas = 0;
        size_t smem = smem_base;
        for (uint32_t j = 0; j < nj; ++j) {
            const uint32_t i = base + j;
            const tn_plan *p = plans[i];
            const uint64_t ld = tn_row_words(ncols[i]);
            tmps[j] = nullptr;
            if (p->resident) continue;  // second pass below
            if (t_last && t_last[i]) {
                tn_internal_count_launches(1);
                order_gate_kernel<<<1, 1, 0, st>>>(p->d_tbounds, t_last[i], p->d_status);
            }
            if (flags & TN_INIT_IDENTITY) {
                if (!src[i]) {
                    tn_internal_count_launches(1);
                    init_identity_kernel<<<grid_for(p->n * 32ull), 256, 0, st>>>(S[i], p->n, ld, p->d_status);
                } else {
                    tn_internal_count_launches(1);
                    zero_kernel<<<grid_for(p->n * ld / 2), 256, 0, st>>>(S[i], (uint64_t)p->n * ld, p->d_status);
                    tn_internal_count_launches(1);
                    init_sources_kernel<<<grid_for(ncols[i]), 256, 0, st>>>(S[i], ld, src[i], ncols[i], p->n,
                                                                            p->d_status);
                }
            }
            if (p->temps) TN_CUDA_TRY(cudaMallocAsync((void **)&tmps[j], p->temps * ld * sizeof(uint64_t), st));
            const size_t need = smem_base + (size_t)p->dcap * p->slab_words * 8;
            if (need > smem) smem = need;
            SlabSplit sp[2];
            const int parts = split_slabs(ld, p->slab_words, p->wave_ctas, sp);
            for (int k = 0; k < parts; ++k) {
                Job &J = jl.job[jl.count++];
                J.blob = p->d_blob;
                J.items = p->d_items;
                J.aux = p->d_aux;
                J.nitems = p->items;
                J.S = S[i];
                J.ld = ld;
                J.tmp = tmps[j];
                J.status = p->d_status;
                J.w_begin = sp[k].w_begin;
                J.sw = sp[k].sw;
                J.cpr = sp[k].sw / 2;
                J.dcap = p->dcap;
                J.cta_begin = ctas;
                ctas += sp[k].ctas;
            }
        }
        // resident-slab jobs after the column-slab ones: their CTAs are short,
        // and the long column-slab CTAs are dispatched first.  Their schedule
        // ring has 8 stages (one CTA of 12 consumer warps per SM) while the
        // resident CTAs fit one wave; beyond that 4, or 2 if only that lets two
        // CTAs share an SM
        uint64_t res_ctas = 0, rb_max = 0;
        for (uint32_t j = 0; j < nj; ++j) {
            const tn_plan *p = plans[base + j];
            if (!p->resident) continue;
            res_ctas += ((ncols[base + j] + 63) / 64 + p->resident - 1) / p->resident;
            const uint64_t rb = kResidentHead + resident_rows_bytes(p->n, p->temps, p->resident);
            if (rb > rb_max) rb_max = rb;
        }
        uint64_t stages = kResidentMaxStages;
        if (res_ctas > (uint64_t)multiprocessors()) {
            stages = 4;
            if (smem <= kHalfSmSmem && rb_max + 4ull * kStageBytes > kHalfSmSmem &&
                rb_max + 2ull * kStageBytes <= kHalfSmSmem)
                stages = 2;
        }
        for (uint32_t j = 0; j < nj; ++j) {
            const uint32_t i = base + j;
            const tn_plan *p = plans[i];
            if (!p->resident) continue;
            const uint64_t ld = tn_row_words(ncols[i]);
            if (t_last && t_last[i]) {
                tn_internal_count_launches(1);
                order_gate_kernel<<<1, 1, 0, st>>>(p->d_tbounds, t_last[i], p->d_status);
            }
            if (flags & TN_INIT_IDENTITY) {
                if (!src[i]) {
                    tn_internal_count_launches(1);
                    init_identity_kernel<<<grid_for(p->n * 32ull), 256, 0, st>>>(S[i], p->n, ld, p->d_status);
                } else {
                    tn_internal_count_launches(1);
                    zero_kernel<<<grid_for(p->n * ld / 2), 256, 0, st>>>(S[i], (uint64_t)p->n * ld, p->d_status);
                    tn_internal_count_launches(1);
                    init_sources_kernel<<<grid_for(ncols[i]), 256, 0, st>>>(S[i], ld, src[i], ncols[i], p->n,
                                                                            p->d_status);
                }
            }
            // words holding columns (the rest of the row is zero padding and stays so)
            const uint64_t used = (ncols[i] + 63) / 64;
            const uint32_t rw = p->resident;
            const uint64_t rb = kResidentHead + resident_rows_bytes(p->n, p->temps, rw);
            uint64_t need = rb + stages * kStageBytes;
            if (need > smem_limit) need = smem_limit;
            if (rb + (uint64_t)kResidentMinStages * kStageBytes > smem_limit) return TN_EINVAL;
            if (need > smem) smem = need;
            Job &J = jl.job[jl.count++];
            J.blob = p->d_blob;
            J.items = p->d_items;
            J.aux = p->d_aux;
            J.nitems = p->items;
            J.S = S[i];
            J.ld = ld;
            J.tmp = nullptr;
            J.status = p->d_status;
            J.w_begin = 0;
            J.sw = rw;
            J.cpr = 0;
            J.dcap = 0;
            J.rw = rw;
            J.rows = p->n;
            J.ntemp = (uint32_t)p->temps;
            J.blob8 = p->blob8;
            J.cta_begin = ctas;
            ctas += (uint32_t)((used + rw - 1) / rw);
        }
        jl.smem_bytes = (uint32_t)smem;
        TN_CUDA_TRY(cudaGetLastError());
        if (ctas) {
            tn_internal_count_launches(1);
            const void *kernel = (flags & kApplyMax) ? (const void *)stream_kernel<true> : (const void *)stream_kernel<false>;
            TN_CUDA_TRY(tn_internal_allow_max_dyn_smem(kernel));
            // 4 consumer warps if two CTAs of that size fit on an SM, else 12
            int pair = 0;
            const int shared_threads = 32 * kWarpsShared + 32;
            TN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pair, kernel, shared_threads, smem));
            const int threads = pair >= 2 ? shared_threads : kMaxThreads;
            if (flags & kApplyMax)
                stream_kernel<true><<<ctas, threads, smem, st>>>(jl);
            else
                stream_kernel<false><<<ctas, threads, smem, st>>>(jl);
        }
        TN_CUDA_TRY(cudaGetLastError());
        for (uint32_t j = 0; j < nj; ++j) {
            const uint32_t i = base + j;
            if (t_last && t_last[i]) {
                tn_internal_count_launches(1);
                set_t_last_kernel<<<1, 1, 0, st>>>(plans[i]->d_tbounds, t_last[i], plans[i]->d_status);
            }
            if (tmps[j]) TN_CUDA_TRY(cudaFreeAsync(tmps[j], st));
        }
        TN_CUDA_TRY(cudaGetLastError());
    }
    return TN_OK;
}

}  // namespace tn

using namespace tn;

extern "C" tn_status tn_plan_apply(const tn_plan *plan, uint64_t *S, uint32_t ncols, const uint32_t *src,
                                   int64_t *t_last, uint32_t flags, void *stream)
{
    if (!plan || !S || (flags & ~TN_INIT_IDENTITY)) return TN_EINVAL;
    return apply_jobs(&plan, &S, &ncols, &src, &t_last, 1, flags, (cudaStream_t)stream);
}

extern "C" tn_status tn_plan_apply_batch(const tn_plan *const *plans, uint64_t *const *S, const uint32_t *ncols,
                                         const uint32_t *const *src, uint32_t count, uint32_t flags, void *stream)
{
    if (!plans || !S || !ncols || count == 0 || (flags & ~TN_INIT_IDENTITY)) return TN_EINVAL;
    if (src) return apply_jobs(plans, S, ncols, src, nullptr, count, flags, (cudaStream_t)stream);
    const uint32_t **none = (const uint32_t **)calloc(count, sizeof(uint32_t *));
    if (!none) return TN_ENOMEM;
    tn_status rc = apply_jobs(plans, S, ncols, none, nullptr, count, flags, (cudaStream_t)stream);
    free(none);
    return rc;
}

// reversed sequence (Section 3.4): event m-1-e becomes event e and its time is
// complemented (~t = -t - 1 keeps equal times equal and the order non-decreasing)
// Directed events are also turned around (u -> v becomes v -> u), so that in
// both modes row i ends as the out-component of i.
__global__ void reverse_events_kernel(const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t m,
                                      bool turn, uint32_t *ru, uint32_t *rv, int64_t *rt)
{
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t s = m - 1 - e;
        ru[e] = turn ? v[s] : u[s];
        rv[e] = turn ? u[s] : v[s];
        rt[e] = ~t[s];
    }
}

static tn_status one_shot(const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t m, uint32_t n,
                          const uint32_t *src, uint32_t ncols, uint64_t *S, int64_t *t_last, uint32_t flags,
                          void *stream);

tn_status tn::reversed_events(const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t m, bool turn,
                              uint32_t **ru, uint32_t **rv, int64_t **rt, cudaStream_t st)
{
    *ru = nullptr;
    *rv = nullptr;
    *rt = nullptr;
    TN_CUDA_TRY(cudaMallocAsync((void **)ru, m * 4, st));
    TN_CUDA_TRY(cudaMallocAsync((void **)rv, m * 4, st));
    TN_CUDA_TRY(cudaMallocAsync((void **)rt, m * 8, st));
    tn_internal_count_launches(1);
    reverse_events_kernel<<<grid_for(m), 256, 0, st>>>(u, v, t, m, turn, *ru, *rv, *rt);
    TN_CUDA_TRY(cudaGetLastError());
    return TN_OK;
}

// TN_REVERSE: the same path over the reversed sequence, from the identity
static tn_status one_shot_reversed(const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t m, uint32_t n,
                                   const uint32_t *src, uint32_t ncols, uint64_t *S, int64_t *t_last,
                                   uint32_t flags, void *stream)
{
    if (t_last || !(flags & TN_INIT_IDENTITY)) return TN_EINVAL;  // not a streaming mode
    if (m == 0) return one_shot(u, v, t, m, n, src, ncols, S, nullptr, flags & ~TN_REVERSE, stream);
    if (!u || !v || !t || m >= (1ull << 30)) return TN_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *ru = nullptr, *rv = nullptr;
    int64_t *rt = nullptr;
    const tn_status rr = reversed_events(u, v, t, m, (flags & TN_DIRECTED) != 0, &ru, &rv, &rt, st);
    if (rr != TN_OK) return rr;
    const tn_status rc = one_shot(ru, rv, rt, m, n, src, ncols, S, nullptr, flags & ~TN_REVERSE, stream);
    cudaFreeAsync(ru, st);
    cudaFreeAsync(rv, st);
    cudaFreeAsync(rt, st);
    return rc;
}

static tn_status one_shot(const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t m, uint32_t n,
                          const uint32_t *src, uint32_t ncols, uint64_t *S, int64_t *t_last, uint32_t flags,
                          void *stream)
{
    if (!S || n == 0 || n >= (1u << 30) || (flags & ~(TN_INIT_IDENTITY | TN_REVERSE | TN_DIRECTED))) return TN_EINVAL;
    if (flags & TN_REVERSE) return one_shot_reversed(u, v, t, m, n, src, ncols, S, t_last, flags, stream);
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t ld = tn_row_words(ncols);
    if (src && (flags & TN_INIT_IDENTITY)) {
        const tn_status rc = validate_sources(src, ncols, n, st);
        if (rc != TN_OK) return rc;
    }
    if (m == 0) {
        if (flags & TN_INIT_IDENTITY) {
            int32_t *zero = nullptr;
            TN_CUDA_TRY(cudaMallocAsync((void **)&zero, sizeof(int32_t), st));
            TN_CUDA_TRY(cudaMemsetAsync(zero, 0, sizeof(int32_t), st));
            if (!src) {
                tn_internal_count_launches(1);
                init_identity_kernel<<<grid_for(n * 32ull), 256, 0, st>>>(S, n, ld, zero);
            } else {
                tn_internal_count_launches(1);
                zero_kernel<<<grid_for(n * ld / 2), 256, 0, st>>>(S, (uint64_t)n * ld, zero);
                tn_internal_count_launches(1);
                init_sources_kernel<<<grid_for(ncols), 256, 0, st>>>(S, ld, src, ncols, n, zero);
            }
            TN_CUDA_TRY(cudaFreeAsync(zero, st));
            TN_CUDA_TRY(cudaGetLastError());
        }
        return TN_OK;
    }
    tn_plan_options opt;
    memset(&opt, 0, sizeof(opt));
    opt.directed = (flags & TN_DIRECTED) ? 1u : 0u;
    tn_plan *plan = nullptr;
    tn_status rc = tn_plan_create(u, v, t, m, n, t_last, &opt, stream, &plan);
    if (rc != TN_OK) return rc;
    flags &= ~TN_DIRECTED;
    rc = apply_jobs((const tn_plan *const *)&plan, &S, &ncols, &src, &t_last, 1, flags, st);
    tn_plan_destroy(plan, stream);
    return rc;
}

extern "C" tn_status tn_component_matrix(const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t m,
                                         uint32_t n, uint64_t *S, int64_t *t_last, uint32_t flags, void *stream)
{
    return one_shot(u, v, t, m, n, nullptr, n, S, t_last, flags, stream);
}

extern "C" tn_status tn_component_columns(const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t m,
                                          uint32_t n, const uint32_t *src, uint32_t nsrc, uint64_t *S,
                                          int64_t *t_last, uint32_t flags, void *stream)
{
    if (!src || nsrc == 0) return TN_EINVAL;
    return one_shot(u, v, t, m, n, src, nsrc, S, t_last, flags, stream);
}

extern "C" tn_status tn_init_matrix(uint64_t *S, uint32_t n_rows, uint32_t ncols, const uint32_t *src, void *stream)
{
    if (!S || n_rows == 0 || ncols == 0 || n_rows >= (1u << 30)) return TN_EINVAL;
    if (!src && ncols != n_rows) return TN_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (src) {
        const tn_status rc = validate_sources(src, ncols, n_rows, st);
        if (rc != TN_OK) return rc;
    }
    const uint64_t ld = tn_row_words(ncols);
    int32_t *zero = nullptr;
    TN_CUDA_TRY(cudaMallocAsync((void **)&zero, sizeof(int32_t), st));
    TN_CUDA_TRY(cudaMemsetAsync(zero, 0, sizeof(int32_t), st));
    if (!src) {
        tn_internal_count_launches(1);
        init_identity_kernel<<<grid_for(n_rows * 32ull), 256, 0, st>>>(S, n_rows, ld, zero);
    } else {
        tn_internal_count_launches(2);
        zero_kernel<<<grid_for(n_rows * ld / 2), 256, 0, st>>>(S, (uint64_t)n_rows * ld, zero);
        init_sources_kernel<<<grid_for(ncols), 256, 0, st>>>(S, ld, src, ncols, n_rows, zero);
    }
    TN_CUDA_TRY(cudaGetLastError());
    TN_CUDA_TRY(cudaFreeAsync(zero, st));
    return TN_OK;
}

extern "C" tn_status tn_selftest_wait_timeout(void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *d = nullptr, h = 0;
    TN_CUDA_TRY(cudaMallocAsync((void **)&d, sizeof(int32_t), st));
    TN_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(int32_t), st));
    tn_internal_count_launches(1);
    wait_selftest_kernel<<<1, 32, 0, st>>>(d);
    TN_CUDA_TRY(cudaGetLastError());
    TN_CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    TN_CUDA_TRY(cudaFreeAsync(d, st));
    TN_CUDA_TRY(cudaStreamSynchronize(st));
    return (tn_status)h;
}

extern "C" uint32_t tn_resident_max_rows(uint32_t resident_words) { return tn::resident_max_rows(resident_words); }
