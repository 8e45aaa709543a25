// Scheduling of an event batch for the column-slab streaming kernel.
//
// Algorithm 1 (Section 3.1) is a strict sequence of row updates, but two
// events that share no node commute, and the columns of the matrix are
// independent.  The schedule groups the updates into "levels": inside a level
// no two updates conflict, so the streaming kernel can issue all of a level's
// row loads at once and only needs a barrier between levels.
//
// Equal timestamps (Section 2.1: adjacency needs dt > 0) are applied as one
// snapshot.  Inside a group G with node counts c(x) (occurrences of x in G):
//   * an event whose two ends both occur once in G is an ordinary update
//     (EVENT: r = S[u] | S[v] into both rows);
//   * a node y occurring once, whose partner x occurs several times, gets
//     ONEWAY: S[y] |= S[x] at level L (x is not written at level L);
//   * a node x occurring several times gets one PULL at level L+1:
//     S[x] |= OR of its partners' rows, where a partner y occurring once is
//     read from S[y] (already y_old | x_old: the extra x_old is harmless) and a
//     partner z occurring several times is read from a saved copy of z's old
//     row (COPY at level L into a temporary slot).
// This reproduces S_new[x] = S_old[x] | OR_{(x,y) in G} S_old[y] exactly.
//
// The batch is cut into windows of about `window_events` events, never inside
// a timestamp group.  Each window is scheduled independently by one CTA
// (levels restart at every window, which acts as one extra barrier):
//   1. node ids of the window are compacted through a hash table;
//   2. one thread scans the window's groups in time order and assigns levels
//      (level of an update = 1 + last level at which any of its rows was
//      touched), tie-group roles, PULL source lists and COPY slots;
//   3. the window's updates are counting-sorted by level.
// A final pass concatenates the windows into one level-ordered op list.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "tn_internal.cuh"

namespace tn {

constexpr int kPlanThreads = 256;
constexpr uint32_t kDefaultWindow = 640;
constexpr uint32_t kDefaultSlab = 16;
constexpr uint32_t kRowBufferBytes = 160 * 1024;  // default shared-memory row buffer, slabs of up to 16 words
constexpr uint32_t kRowBufferWide = 192 * 1024;   // default (and largest) row buffer for wider slabs
constexpr uint32_t kWinFields = 8;  // nops, nlev, naux, ntemp, local, blob8, nitems, all ops
constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr uint32_t kNone = 0xFFFFFFFFu;

// event flags stored in the grp array once scheduling is done
constexpr uint32_t kFlagDir = 1u << 27;   // directed event outside a tie group: one ONEWAY
constexpr uint32_t kFlagNoop = 1u << 28;
constexpr uint32_t kFlagIso = 1u << 29;
constexpr uint32_t kFlagShA = 1u << 30;
constexpr uint32_t kFlagShB = 1u << 31;

// arena layout (uint32 words) for a window of E events:
//   lu[E] lv[E] grp[E] evl[E] run_node[E] run_aux[E] run_lev[E] run_temp[E] rowsg[2E] scratch
// scratch: hash keys + ids (2*H words, H = hash slots) during id assignment,
// then node state nlev/ncnt/nrun (3*D words, D <= 2E distinct nodes), then the
// level histogram (<= 2E + 3 words).
__host__ __device__ inline uint64_t hash_slots(uint64_t E) { return ((3 * E + 31) / 32) * 32; }
__host__ __device__ inline uint64_t arena_words(uint64_t E)
{
    const uint64_t H = hash_slots(E);
    uint64_t scratch = 2 * H;
    if (6 * E > scratch) scratch = 6 * E;
    if (2 * E + 3 > scratch) scratch = 2 * E + 3;
    return 10 * E + scratch;
}

struct PlanArgs {
    const uint32_t *u, *v;
    const int64_t *t;
    uint64_t m;
    uint32_t n;
    const int64_t *t_after;
    uint32_t window;     // target events per window
    uint32_t directed;   // 1: events are u -> v (only S[v] is updated)
    uint32_t nw;         // number of windows
    uint64_t *wstart;    // [nw + 1]
    uint32_t smem_max_events;
    uint32_t dcap;          // row slots of a local window
    uint32_t max_rec_words; // largest local record (words)
    // per-window results (kWinFields each)
    uint32_t *wcount;    // [kWinFields * nw]
    // staging (window w uses the regions starting at 3*s_w / 2*s_w + w / 10*s_w + 8*w)
    uint2 *ops_stage;    // [3m]
    uint32_t *aux_stage; // [3m]
    uint32_t *lvl_stage; // [2m + nw + 1]
    uint32_t *rec_stage; // [10m + 8nw]
    // large windows
    uint32_t *big_list;  // [nw]
    uint64_t *big_off;   // [nw]
    uint32_t *big_arena;
    // global counters: [0] error flags, [1] number of big windows, [2] arena words of
    // the big windows, [3] largest window scheduled in shared memory
    unsigned long long *counters;
};

// ---------------------------------------------------------------------------
// validation (Section 2.1: nodes in [0, n), events time-ordered)
// ---------------------------------------------------------------------------
__global__ void validate_kernel(PlanArgs a)
{
    uint32_t bad = 0;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < a.m;
         e += (uint64_t)gridDim.x * blockDim.x) {
        if (a.u[e] >= a.n || a.v[e] >= a.n) bad |= 1u;
        if (e > 0 && a.t[e] < a.t[e - 1]) bad |= 2u;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.t_after && a.m > 0 && !(a.t[0] > *a.t_after)) bad |= 2u;
    if (bad) atomicOr(&a.counters[0], (unsigned long long)bad);
}

// window w starts at the first timestamp-group start at or after w * window
__global__ void window_kernel(PlanArgs a)
{
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w <= a.nw;
         w += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t s;
        if (w == 0) {
            s = 0;
        } else if (w == a.nw) {
            s = a.m;
        } else {
            s = w * (uint64_t)a.window;
            if (s >= a.m) {
                s = a.m;
            } else if (a.t[s] == a.t[s - 1]) {
                // first index with t > t[s] (upper bound) by binary search
                const int64_t key = a.t[s];
                uint64_t lo = s, hi = a.m;
                while (lo < hi) {
                    uint64_t mid = lo + (hi - lo) / 2;
                    if (a.t[mid] > key) hi = mid;
                    else lo = mid + 1;
                }
                s = lo;
            }
        }
        a.wstart[w] = s;
    }
}

__global__ void big_window_kernel(PlanArgs a)
{
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < a.nw;
         w += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t E = a.wstart[w + 1] - a.wstart[w];
        if (E <= a.smem_max_events) atomicMax(&a.counters[3], (unsigned long long)E);
        if (E > a.smem_max_events) {
            unsigned long long slot = atomicAdd(&a.counters[1], 1ull);
            unsigned long long off = atomicAdd(&a.counters[2], (unsigned long long)arena_words(E));
            a.big_list[slot] = (uint32_t)w;
            a.big_off[slot] = off;
        }
    }
}

// ---------------------------------------------------------------------------
// per-window scheduler
// ---------------------------------------------------------------------------
__device__ inline uint32_t hslot(uint32_t key, uint32_t H)
{
    return (uint32_t)(((uint64_t)(key * 0x9E3779B1u) * H) >> 32);
}

__device__ inline void hinsert(uint32_t *hkey, uint32_t H, uint32_t key)
{
    uint32_t s = hslot(key, H);
    for (uint32_t probe = 0; probe < H; ++probe) {  // the table always has free slots
        uint32_t cur = hkey[s];
        if (cur == key) return;
        if (cur == kEmpty) {
            uint32_t prev = atomicCAS(&hkey[s], kEmpty, key);
            if (prev == kEmpty || prev == key) return;
        }
        s = (s + 1 == H) ? 0 : s + 1;
    }
}

__device__ inline uint32_t hlookup(const uint32_t *hkey, const uint32_t *hval, uint32_t H, uint32_t key)
{
    uint32_t s = hslot(key, H);
    for (uint32_t probe = 0; probe < H && hkey[s] != key; ++probe) s = (s + 1 == H) ? 0 : s + 1;
    return hval[s];
}

// Timestamp groups of at least this many events are scheduled by the whole CTA.
constexpr uint32_t kParGroup = 128;
constexpr uint32_t kClaim = 0xFFFFFFFEu;  // run / temp slot being assigned

// Scan state shared by the threads of a window's CTA: nruns, naux, ntemp,
// maxlev, next event, end of the large group at it.
enum { kScRuns = 0, kScAux, kScTemp, kScMaxlev, kScNext, kScEnd, kScCount };

// The snapshot rule for one large undirected timestamp group [i, g1), with
// every thread of the CTA.  It yields the same roles, levels, runs (PULLs),
// saved-row slots and source lists as the sequential scan; only the numbering
// of runs and slots and the order of ops inside a level and of sources inside
// a PULL list may differ, and none of them changes the result.  Nodes that
// occur once in the group take part in exactly one event, so a lone event
// (both ends once) touches no other event's rows and gets its level at once;
// the other events share one level L = 1 + the latest level of their nodes,
// with the PULLs at L + 1.  Phases are separated by barriers, so a run's
// and a slot's number are final before anyone reads them.
__device__ void schedule_group_parallel(uint32_t i, uint32_t g1, const uint32_t *lu, const uint32_t *lv,
                                        uint32_t *grp, uint32_t *evl, uint32_t *run_node, uint32_t *run_aux,
                                        uint32_t *run_lev, uint32_t *run_temp, uint32_t *nlev, uint32_t *ncnt,
                                        uint32_t *nrun, uint32_t *auxw, uint32_t *sc)
{
    __shared__ uint32_t Lc, any, run0;
    const uint32_t T = blockDim.x, tid = threadIdx.x;
    for (uint32_t j = i + tid; j < g1; j += T) {
        ncnt[lu[j]] = 0;
        ncnt[lv[j]] = 0;
        nrun[lu[j]] = kNone;
        nrun[lv[j]] = kNone;
    }
    if (tid == 0) {
        Lc = 0;
        any = 0;
        run0 = sc[kScRuns];
    }
    __syncthreads();
    for (uint32_t j = i + tid; j < g1; j += T)
        if (lu[j] != lv[j]) {
            atomicAdd(&ncnt[lu[j]], 1u);
            atomicAdd(&ncnt[lv[j]], 1u);
        }
    __syncthreads();
    // roles; lone events' levels; one run (PULL) per node occurring several times
    auto claim_run = [&](uint32_t x) {
        if (atomicCAS(&nrun[x], kNone, kClaim) != kNone) return;
        const uint32_t r = atomicAdd(&sc[kScRuns], 1u);
        const uint32_t b = atomicAdd(&sc[kScAux], 1u + ncnt[x]);
        run_node[r] = x;
        run_aux[r] = b;
        run_lev[r] = 0;  // fill counter until the level is known
        run_temp[r] = kNone;
        auxw[b] = ncnt[x];
        nrun[x] = r;
    };
    for (uint32_t j = i + tid; j < g1; j += T) {
        const uint32_t x = lu[j], y = lv[j];
        if (x == y) {
            grp[j] = kFlagNoop;
            continue;
        }
        const bool sx = ncnt[x] > 1, sy = ncnt[y] > 1;
        if (!sx && !sy) {
            const uint32_t L = 1 + max(nlev[x], nlev[y]);
            nlev[x] = L;
            nlev[y] = L;
            evl[j] = L;
            grp[j] = kFlagIso;
            atomicMax(&sc[kScMaxlev], L);
            continue;
        }
        atomicMax(&Lc, max(nlev[x], nlev[y]));
        any = 1;
        grp[j] = (sx ? kFlagShA : 0u) | (sy ? kFlagShB : 0u);
        if (sx) claim_run(x);
        if (sy) claim_run(y);
    }
    __syncthreads();
    // saved rows: a node occurring several times whose partner does too is
    // read from a copy of its old row
    auto claim_temp = [&](uint32_t r) {
        if (atomicCAS(&run_temp[r], kNone, kClaim) == kNone) run_temp[r] = atomicAdd(&sc[kScTemp], 1u);
    };
    for (uint32_t j = i + tid; j < g1; j += T)
        if (grp[j] == (kFlagShA | kFlagShB)) {
            claim_temp(nrun[lu[j]]);
            claim_temp(nrun[lv[j]]);
        }
    __syncthreads();
    // source lists
    for (uint32_t j = i + tid; j < g1; j += T) {
        const uint32_t f = grp[j];
        if (f & (kFlagNoop | kFlagIso)) continue;
        const uint32_t x = lu[j], y = lv[j];
        if (f == (kFlagShA | kFlagShB)) {
            const uint32_t rx = nrun[x], ry = nrun[y];
            auxw[run_aux[rx] + 1 + atomicAdd(&run_lev[rx], 1u)] = kTempRef | run_temp[ry];
            auxw[run_aux[ry] + 1 + atomicAdd(&run_lev[ry], 1u)] = kTempRef | run_temp[rx];
        } else if (f & kFlagShA) {
            const uint32_t rx = nrun[x];
            auxw[run_aux[rx] + 1 + atomicAdd(&run_lev[rx], 1u)] = y;
        } else {
            const uint32_t ry = nrun[y];
            auxw[run_aux[ry] + 1 + atomicAdd(&run_lev[ry], 1u)] = x;
        }
    }
    __syncthreads();
    // levels of the shared part: ONEWAY / COPY at L, PULL at L + 1
    if (any) {
        const uint32_t L = Lc + 1;
        for (uint32_t j = i + tid; j < g1; j += T) {
            if (grp[j] & (kFlagNoop | kFlagIso)) continue;
            evl[j] = L;
            nlev[lu[j]] = L + 1;
            nlev[lv[j]] = L + 1;
        }
        for (uint32_t r = run0 + tid; r < sc[kScRuns]; r += T) run_lev[r] = L;
        if (tid == 0) atomicMax(&sc[kScMaxlev], L + 1);
    }
    __syncthreads();
}

__device__ void schedule_window(const PlanArgs &a, uint32_t w, uint32_t *arena)
{
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t tot;
    __shared__ uint32_t res[8];  // nops, maxlev, naux, ntemp, nruns, local, nitems

    const uint64_t s = a.wstart[w];
    const uint32_t E = (uint32_t)(a.wstart[w + 1] - s);
    uint32_t *cnt = a.wcount + (uint64_t)kWinFields * w;
    if (E == 0) {
        if (threadIdx.x < kWinFields) cnt[threadIdx.x] = 0;
        return;
    }
    const uint32_t T = blockDim.x, tid = threadIdx.x;
    const uint32_t H = (uint32_t)hash_slots(E);
    uint32_t *lu = arena, *lv = lu + E, *grp = lv + E, *evl = grp + E;
    uint32_t *run_node = evl + E, *run_aux = run_node + E, *run_lev = run_aux + E, *run_temp = run_lev + E;
    uint32_t *rowsg = run_temp + E;  // [2E] global id of every local row id
    uint32_t *scratch = rowsg + 2 * E;
    uint32_t *hkey = scratch, *hval = scratch + H;
    const uint32_t *U = a.u + s, *V = a.v + s;
    const int64_t *Tt = a.t + s;

    // 1. compact node ids (local row ids 0..D-1)
    for (uint32_t i = tid; i < H; i += T) hkey[i] = kEmpty;
    __syncthreads();
    for (uint32_t i = tid; i < E; i += T) {
        hinsert(hkey, H, U[i]);
        hinsert(hkey, H, V[i]);
    }
    __syncthreads();
    for (uint32_t i = tid; i < H; i += T) hval[i] = hkey[i] != kEmpty ? 1u : 0u;
    __syncthreads();
    const uint32_t D = block_excl_scan_array(hval, H, warp_sums, &tot);
    for (uint32_t i = tid; i < H; i += T)
        if (hkey[i] != kEmpty) rowsg[hval[i]] = hkey[i];
    for (uint32_t i = tid; i < E; i += T) {
        lu[i] = hlookup(hkey, hval, H, U[i]);
        lv[i] = hlookup(hkey, hval, H, V[i]);
        grp[i] = (i == 0 || Tt[i] != Tt[i - 1]) ? 1u : 0u;
    }
    __syncthreads();
    block_excl_scan_array(grp, E, warp_sums, &tot);  // grp[i] = starts before i
    for (uint32_t i = tid; i < E; i += T) grp[i] += (i == 0 || Tt[i] != Tt[i - 1]) ? 1u : 0u;
    // grp[i] is now 1 + group index, which is all the scan below needs.
    uint32_t *nlev = scratch, *ncnt = scratch + D, *nrun = scratch + 2 * D;
    __syncthreads();
    for (uint32_t i = tid; i < D; i += T) {
        nlev[i] = 0;
        ncnt[i] = 0;
        nrun[i] = kNone;
    }
    __syncthreads();

    // 2. level scan in time order: one thread takes the groups one by one and
    //    hands every large undirected group to the whole CTA.  Rows are named
    //    by local ids here; PULL source lists hold local ids or temp references.
    __shared__ uint32_t sc[kScCount];
    if (tid == 0)
        for (int q = 0; q < kScCount; ++q) sc[q] = 0;
    __syncthreads();
    for (;;) {
    if (tid == 0) {
        uint32_t nruns = sc[kScRuns], naux = sc[kScAux], ntemp = sc[kScTemp], maxlev = sc[kScMaxlev];
        uint32_t *auxw = a.aux_stage + 3 * s;
        uint32_t i = sc[kScNext];
        while (i < E && a.directed) {
            // directed events x -> y: only y is written.  A lone event is one
            // ONEWAY y |= x; a tie group becomes one PULL per receiver (level
            // L+1) over its senders' rows, a sender that also receives in the
            // group being read from a copy saved at level L.
            const uint32_t g = grp[i];
            uint32_t g1 = i + 1;
            while (g1 < E && grp[g1] == g) ++g1;
            if (g1 == i + 1) {
                const uint32_t x = lu[i], y = lv[i];
                if (x == y) {
                    grp[i] = kFlagNoop;
                } else {
                    const uint32_t L = 1 + max(nlev[x], nlev[y]);
                    nlev[x] = L;
                    nlev[y] = L;
                    evl[i] = L;
                    grp[i] = kFlagDir;
                    maxlev = max(maxlev, L);
                }
                i = g1;
                continue;
            }
            for (uint32_t j = i; j < g1; ++j) {
                ncnt[lv[j]] = 0;
                nrun[lu[j]] = kNone;
                nrun[lv[j]] = kNone;
            }
            uint32_t Lc = 0;
            bool any = false;
            for (uint32_t j = i; j < g1; ++j) {
                if (lu[j] == lv[j]) continue;
                ++ncnt[lv[j]];
                Lc = max(Lc, max(nlev[lu[j]], nlev[lv[j]]));
            }
            const uint32_t run0 = nruns;
            for (uint32_t j = i; j < g1; ++j) {  // one run per receiver
                const uint32_t y = lv[j];
                if (lu[j] == y || nrun[y] != kNone) continue;
                const uint32_t ry = nruns++;
                nrun[y] = ry;
                run_node[ry] = y;
                run_aux[ry] = naux;
                run_lev[ry] = 0;  // fill counter until the level is known
                run_temp[ry] = kNone;
                auxw[naux] = ncnt[y];
                naux += 1 + ncnt[y];
            }
            for (uint32_t j = i; j < g1; ++j) {
                const uint32_t x = lu[j], y = lv[j];
                if (x == y) {
                    grp[j] = kFlagNoop;
                    continue;
                }
                any = true;
                grp[j] = kFlagShA | kFlagShB;  // no op of its own: the receiver's PULL covers it
                uint32_t ref = x;
                const uint32_t rx = nrun[x];
                if (rx != kNone) {  // x also receives in this group: read its saved old row
                    if (run_temp[rx] == kNone) run_temp[rx] = ntemp++;
                    ref = kTempRef | run_temp[rx];
                }
                const uint32_t ry = nrun[y];
                auxw[run_aux[ry] + 1 + run_lev[ry]++] = ref;
            }
            if (any) {
                const uint32_t L = Lc + 1;
                for (uint32_t j = i; j < g1; ++j) {
                    if (grp[j] & kFlagNoop) continue;
                    nlev[lu[j]] = L + 1;
                    nlev[lv[j]] = L + 1;
                }
                for (uint32_t r = run0; r < nruns; ++r) run_lev[r] = L;
                maxlev = max(maxlev, L + 1);
            }
            i = g1;
        }
        while (i < E) {
            const uint32_t g = grp[i];
            if (i + kParGroup <= E && grp[i + kParGroup - 1] == g) break;  // a large group: the whole CTA
            uint32_t g1 = i + 1;
            while (g1 < E && grp[g1] == g) ++g1;
            if (g1 == i + 1) {
                const uint32_t x = lu[i], y = lv[i];
                if (x == y) {
                    grp[i] = kFlagNoop;
                } else {
                    const uint32_t L = 1 + max(nlev[x], nlev[y]);
                    nlev[x] = L;
                    nlev[y] = L;
                    evl[i] = L;
                    grp[i] = kFlagIso;
                    maxlev = max(maxlev, L);
                }
            } else {
                // occurrences of every node inside the group
                for (uint32_t j = i; j < g1; ++j) {
                    ncnt[lu[j]] = 0;
                    ncnt[lv[j]] = 0;
                    nrun[lu[j]] = kNone;
                    nrun[lv[j]] = kNone;
                }
                for (uint32_t j = i; j < g1; ++j) {
                    if (lu[j] == lv[j]) continue;
                    ++ncnt[lu[j]];
                    ++ncnt[lv[j]];
                }
                const uint32_t run0 = nruns;
                uint32_t Lc = 0;
                bool any = false;
                for (uint32_t j = i; j < g1; ++j) {
                    const uint32_t x = lu[j], y = lv[j];
                    if (x == y) {
                        grp[j] = kFlagNoop;
                        continue;
                    }
                    const bool sx = ncnt[x] > 1, sy = ncnt[y] > 1;
                    if (!sx && !sy) {
                        const uint32_t L = 1 + max(nlev[x], nlev[y]);
                        nlev[x] = L;
                        nlev[y] = L;
                        evl[j] = L;
                        grp[j] = kFlagIso;
                        maxlev = max(maxlev, L);
                        continue;
                    }
                    any = true;
                    Lc = max(Lc, max(nlev[x], nlev[y]));
                    grp[j] = (sx ? kFlagShA : 0u) | (sy ? kFlagShB : 0u);
                    uint32_t rx = kNone, ry = kNone;
                    if (sx) {
                        rx = nrun[x];
                        if (rx == kNone) {
                            rx = nruns++;
                            nrun[x] = rx;
                            run_node[rx] = x;
                            run_aux[rx] = naux;
                            run_lev[rx] = 0;  // fill counter until the level is known
                            run_temp[rx] = kNone;
                            auxw[naux] = ncnt[x];
                            naux += 1 + ncnt[x];
                        }
                    }
                    if (sy) {
                        ry = nrun[y];
                        if (ry == kNone) {
                            ry = nruns++;
                            nrun[y] = ry;
                            run_node[ry] = y;
                            run_aux[ry] = naux;
                            run_lev[ry] = 0;
                            run_temp[ry] = kNone;
                            auxw[naux] = ncnt[y];
                            naux += 1 + ncnt[y];
                        }
                    }
                    if (sx && sy) {
                        if (run_temp[rx] == kNone) run_temp[rx] = ntemp++;
                        if (run_temp[ry] == kNone) run_temp[ry] = ntemp++;
                        auxw[run_aux[rx] + 1 + run_lev[rx]++] = kTempRef | run_temp[ry];
                        auxw[run_aux[ry] + 1 + run_lev[ry]++] = kTempRef | run_temp[rx];
                    } else if (sx) {
                        auxw[run_aux[rx] + 1 + run_lev[rx]++] = y;
                    } else {
                        auxw[run_aux[ry] + 1 + run_lev[ry]++] = x;
                    }
                }
                if (any) {
                    const uint32_t L = Lc + 1;
                    for (uint32_t j = i; j < g1; ++j) {
                        const uint32_t f = grp[j];
                        if (f & (kFlagNoop | kFlagIso)) continue;
                        evl[j] = L;
                        nlev[lu[j]] = L + 1;
                        nlev[lv[j]] = L + 1;
                    }
                    for (uint32_t r = run0; r < nruns; ++r) run_lev[r] = L;
                    maxlev = max(maxlev, L + 1);
                }
            }
            i = g1;
        }
        sc[kScRuns] = nruns;
        sc[kScAux] = naux;
        sc[kScTemp] = ntemp;
        sc[kScMaxlev] = maxlev;
        sc[kScNext] = i;
        if (i < E) {  // end of the large group at i: first index past it (grp is non-decreasing there)
            uint32_t lo = i, hi = E;
            while (lo < hi) {
                const uint32_t mid = lo + (hi - lo) / 2;
                if (grp[mid] > grp[i]) hi = mid;
                else lo = mid + 1;
            }
            sc[kScEnd] = lo;
        }
    }
    __syncthreads();
    if (sc[kScNext] >= E) break;
    schedule_group_parallel(sc[kScNext], sc[kScEnd], lu, lv, grp, evl, run_node, run_aux, run_lev, run_temp, nlev,
                            ncnt, nrun, a.aux_stage + 3 * s, sc);
    if (tid == 0) sc[kScNext] = sc[kScEnd];
    __syncthreads();
    }
    if (tid == 0) {
        res[1] = sc[kScMaxlev];
        res[2] = sc[kScAux];
        res[3] = sc[kScTemp];
        res[4] = sc[kScRuns];
        res[6] = 0;
    }
    __syncthreads();
    const uint32_t maxlev = res[1], naux = res[2], ntemp = res[3], nruns = res[4];

    // 3. counting sort of the updates by level (levels 1..maxlev -> 0..maxlev-1)
    uint32_t *lh = scratch;  // node state is dead
    for (uint32_t j = tid; j < maxlev + 1; j += T) lh[j] = 0;
    __syncthreads();
    for (uint32_t i = tid; i < E; i += T) {
        const uint32_t f = grp[i];
        if (f & kFlagNoop) continue;
        if (f & (kFlagIso | kFlagDir)) {
            atomicAdd(&lh[evl[i] - 1], 1u);
        } else {
            if (!(f & kFlagShA)) atomicAdd(&lh[evl[i] - 1], 1u);
            if (!(f & kFlagShB)) atomicAdd(&lh[evl[i] - 1], 1u);
        }
    }
    for (uint32_t r = tid; r < nruns; r += T) {
        atomicAdd(&lh[run_lev[r]], 1u);  // PULL at level L+1 -> index L
        if (run_temp[r] != kNone) atomicAdd(&lh[run_lev[r] - 1], 1u);
    }
    __syncthreads();
    const uint32_t nops = block_excl_scan_array(lh, maxlev + 1, warp_sums, &tot);

    // 4. mode: the window's rows and saved rows fit the streaming kernel's
    //    shared-memory row buffer, and its record fits one staging buffer
    const uint32_t rec_words = 4 + D + (maxlev + 1) + nops + naux;
    const uint32_t rec_words_pad = (rec_words + 3u) & ~3u;
    const bool local = D + ntemp <= a.dcap && rec_words_pad <= a.max_rec_words;

    if (local) {
        // record: header | rows[D] | lvl[maxlev+1] | ops[nops] | aux[naux] | pad
        uint32_t *rec = a.rec_stage + 10 * s + 8ull * w;
        uint32_t *rrows = rec + 4, *rlvl = rrows + D, *rops = rlvl + maxlev + 1, *raux = rops + nops;
        if (tid == 0) {
            rec[0] = D;
            rec[1] = ntemp;
            rec[2] = maxlev;
            rec[3] = nops;
        }
        for (uint32_t d = tid; d < D; d += T) rrows[d] = rowsg[d];
        for (uint32_t j = tid; j < maxlev + 1; j += T) rlvl[j] = lh[j];
        for (uint32_t k = rec_words + tid; k < rec_words_pad; k += T) rec[k] = 0;
        const uint32_t *auxw = a.aux_stage + 3 * s;
        for (uint32_t r = tid; r < nruns; r += T) {
            const uint32_t b = run_aux[r], c = auxw[b];
            raux[b] = c;
            for (uint32_t q = 1; q <= c; ++q) {
                const uint32_t ref = auxw[b + q];
                raux[b + q] = (ref & kTempRef) ? D + (ref & ~kTempRef) : ref;
            }
        }
        __syncthreads();
        for (uint32_t i = tid; i < E; i += T) {
            const uint32_t f = grp[i];
            if (f & kFlagNoop) continue;
            const uint32_t x = lu[i], y = lv[i];
            if (f & kFlagDir) {
                rops[atomicAdd(&lh[evl[i] - 1], 1u)] = local_op(kOneway, y, x);  // y |= x
                continue;
            }
            const uint32_t L = evl[i] - 1;
            if (f & kFlagIso) {
                rops[atomicAdd(&lh[L], 1u)] = local_op(kEvent, x, y);
            } else {
                if (!(f & kFlagShA)) rops[atomicAdd(&lh[L], 1u)] = local_op(kOneway, x, y);
                if (!(f & kFlagShB)) rops[atomicAdd(&lh[L], 1u)] = local_op(kOneway, y, x);
            }
        }
        for (uint32_t r = tid; r < nruns; r += T) {
            const uint32_t L = run_lev[r];
            rops[atomicAdd(&lh[L], 1u)] = local_op(kPull, run_node[r], run_aux[r]);
            if (run_temp[r] != kNone) rops[atomicAdd(&lh[L - 1], 1u)] = local_op(kCopy, D + run_temp[r], run_node[r]);
        }
        // last write of every row: ops are in level order and a level writes a
        // row at most once, so it is the op with the highest index writing it
        uint32_t *lastw = scratch + maxlev + 2;  // lh holds scratch[0 .. maxlev]
        for (uint32_t d = tid; d < D; d += T) lastw[d] = 0;
        __syncthreads();
        for (uint32_t i = tid; i < nops; i += T) {
            const uint32_t op = rops[i], kind = op >> kKindShift;
            if (kind == kCopy) continue;  // writes a saved copy, not a row
            atomicMax(&lastw[(op >> kLocalBits) & kLocalMask], i + 1);
            if (kind == kEvent) atomicMax(&lastw[op & kLocalMask], i + 1);
        }
        __syncthreads();
        for (uint32_t i = tid; i < nops; i += T) {
            uint32_t op = rops[i];
            const uint32_t kind = op >> kKindShift;
            if (kind == kCopy) continue;
            if (lastw[(op >> kLocalBits) & kLocalMask] == i + 1) op |= kLastA;
            if (kind == kEvent && lastw[op & kLocalMask] == i + 1) op |= kLastB;
            rops[i] = op;
        }
        if (tid == 0) {
            cnt[0] = 0;
            cnt[1] = maxlev;
            cnt[2] = 0;
            cnt[3] = 0;
            cnt[4] = 1;
            cnt[5] = rec_words_pad / 2;
            cnt[6] = 1;
            cnt[7] = nops;
        }
        return;
    }

    // global mode: ops name rows by node id; PULL lists are converted in place
    uint32_t *lvl_out = a.lvl_stage + 2 * s + w;
    for (uint32_t j = tid; j < maxlev + 1; j += T) lvl_out[j] = lh[j];
    for (uint32_t j = tid; j < maxlev; j += T) {
        const uint32_t c = lh[j + 1] - lh[j];
        atomicAdd(&res[6], (c + kTileOps - 1) / kTileOps);
    }
    uint32_t *auxw = a.aux_stage + 3 * s;
    for (uint32_t r = tid; r < nruns; r += T) {
        const uint32_t b = run_aux[r], c = auxw[b];
        for (uint32_t q = 1; q <= c; ++q) {
            const uint32_t ref = auxw[b + q];
            if (!(ref & kTempRef)) auxw[b + q] = rowsg[ref];
        }
    }
    __syncthreads();
    uint2 *ops = a.ops_stage + 3 * s;
    for (uint32_t i = tid; i < E; i += T) {
        const uint32_t f = grp[i];
        if (f & kFlagNoop) continue;
        const uint32_t x = U[i], y = V[i];
        const uint32_t L = evl[i] - 1;
        if (f & kFlagDir) {
            ops[atomicAdd(&lh[L], 1u)] = make_uint2(op_a(kOneway, y), x);  // y |= x
            continue;
        }
        if (f & kFlagIso) {
            ops[atomicAdd(&lh[L], 1u)] = make_uint2(op_a(kEvent, x), y);
        } else {
            if (!(f & kFlagShA)) ops[atomicAdd(&lh[L], 1u)] = make_uint2(op_a(kOneway, x), y);
            if (!(f & kFlagShB)) ops[atomicAdd(&lh[L], 1u)] = make_uint2(op_a(kOneway, y), x);
        }
    }
    for (uint32_t r = tid; r < nruns; r += T) {
        const uint32_t L = run_lev[r], xg = rowsg[run_node[r]];
        ops[atomicAdd(&lh[L], 1u)] = make_uint2(op_a(kPull, xg), (uint32_t)(3 * s) + run_aux[r]);
        if (run_temp[r] != kNone) ops[atomicAdd(&lh[L - 1], 1u)] = make_uint2(op_a(kCopy, run_temp[r]), xg);
    }
    __syncthreads();
    if (tid == 0) {
        cnt[0] = nops;
        cnt[1] = maxlev;
        cnt[2] = naux;
        cnt[3] = ntemp;
        cnt[4] = 0;
        cnt[5] = (nops + 1u) & ~1u;
        cnt[6] = res[6];
        cnt[7] = nops;
    }
}

__global__ void __launch_bounds__(kPlanThreads) schedule_smem_kernel(PlanArgs a)
{
    extern __shared__ uint32_t smem_arena[];
    const uint32_t w = blockIdx.x;
    const uint64_t E = a.wstart[w + 1] - a.wstart[w];
    if (E > a.smem_max_events) return;  // scheduled by the large-window kernel
    schedule_window(a, w, smem_arena);
}

__global__ void __launch_bounds__(kPlanThreads) schedule_big_kernel(PlanArgs a)
{
    const uint32_t w = a.big_list[blockIdx.x];
    schedule_window(a, w, a.big_arena + a.big_off[blockIdx.x]);
}

// ---------------------------------------------------------------------------
// concatenation of the windows
// ---------------------------------------------------------------------------
struct Totals {
    unsigned long long items, blob8, naux, tmax, levels, ops, local;
};

// exclusive scans over windows of nitems / blob8 / naux (one CTA)
__global__ void window_scan_kernel(const uint32_t *wcount, uint32_t nw, uint64_t *base /* [3*nw] */, Totals *tot)
{
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t total;
    __shared__ unsigned long long carry[3];
    __shared__ unsigned long long levels, ops, local;
    __shared__ unsigned int tmax;
    if (threadIdx.x < 3) carry[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        tmax = 0;
        levels = ops = local = 0;
    }
    __syncthreads();
    static_assert(kWinFields == 8, "two 16-byte loads per window");
    for (uint32_t c0 = 0; c0 < nw; c0 += blockDim.x) {
        const uint32_t w = c0 + threadIdx.x;
        uint4 lo = make_uint4(0u, 0u, 0u, 0u), hi = make_uint4(0u, 0u, 0u, 0u);
        if (w < nw) {
            const uint4 *c = reinterpret_cast<const uint4 *>(wcount + (uint64_t)kWinFields * w);
            lo = c[0];  // nops, nlev, naux, ntemp
            hi = c[1];  // local, blob8, nitems, all ops
        }
        const uint32_t x[3] = {hi.z, hi.y, lo.z};  // items, blob8, naux
        for (int k = 0; k < 3; ++k) {
            uint32_t ex = block_excl_scan_value(x[k], warp_sums, &total);
            if (w < nw) base[3ull * w + k] = carry[k] + ex;
            __syncthreads();
            if (threadIdx.x == 0) carry[k] += total;
            __syncthreads();
        }
        // totals: a warp reduction first, then one shared atomic per warp
        unsigned long long lv = lo.y, op = hi.w, lc = hi.x;
        uint32_t tm = lo.w;
        for (int d = 16; d > 0; d >>= 1) {
            lv += __shfl_xor_sync(0xffffffffu, lv, d);
            op += __shfl_xor_sync(0xffffffffu, op, d);
            lc += __shfl_xor_sync(0xffffffffu, lc, d);
            tm = max(tm, __shfl_xor_sync(0xffffffffu, tm, d));
        }
        if ((threadIdx.x & 31u) == 0) {
            atomicMax(&tmax, tm);
            atomicAdd(&levels, lv);
            atomicAdd(&ops, op);
            atomicAdd(&local, lc);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        tot->items = carry[0];
        tot->blob8 = carry[1];
        tot->naux = carry[2];
        tot->tmax = tmax;
        tot->levels = levels;
        tot->ops = ops;
        tot->local = local;
    }
}

// concatenation of the windows into the blob, the item list and the aux list
__global__ void compact_kernel(PlanArgs a, const uint64_t *base, uint2 *blob, uint4 *items, uint32_t *aux)
{
    const uint32_t w = blockIdx.x;
    if (w >= a.nw) return;
    const uint64_t s = a.wstart[w];
    const uint32_t *c = a.wcount + (uint64_t)kWinFields * w;
    const uint64_t ib = base[3ull * w], bb = base[3ull * w + 1], ab = base[3ull * w + 2];
    if (c[4]) {
        // local record, copied as 8-byte units
        const uint2 *src = reinterpret_cast<const uint2 *>(a.rec_stage + 10 * s + 8ull * w);
        for (uint32_t k = threadIdx.x; k < c[5]; k += blockDim.x) blob[bb + k] = src[k];
        if (threadIdx.x == 0) items[ib] = make_uint4((uint32_t)bb, c[5], kItemLocal, 0u);
        return;
    }
    const uint32_t nops = c[0], nlev = c[1], naux = c[2];
    if (nops == 0) return;
    const uint2 *os = a.ops_stage + 3 * s;
    for (uint32_t k = threadIdx.x; k < nops; k += blockDim.x) {
        uint2 op = os[k];
        if ((op.x >> kKindShift) == kPull) op.y = (uint32_t)(op.y - 3 * s + ab);
        blob[bb + k] = op;
    }
    const uint32_t *as = a.aux_stage + 3 * s;
    for (uint32_t k = threadIdx.x; k < naux; k += blockDim.x) aux[ab + k] = as[k];
    if (threadIdx.x == 0) {
        const uint32_t *ls = a.lvl_stage + 2 * s + w;
        uint64_t it = ib;
        for (uint32_t l = 0; l < nlev; ++l) {
            const uint32_t b = ls[l], e = ls[l + 1];
            for (uint32_t q = b; q < e; q += kTileOps) {
                const uint32_t qe = min(e, q + kTileOps);
                items[it++] = make_uint4((uint32_t)(bb + q), qe - q, qe == e ? kItemLevelEnd : 0u, 0u);
            }
        }
    }
}

// the batch's time bounds, known on the host, into the plan (no read of t, so
// the caller may free the events as soon as tn_plan_create returns)
__global__ void tbounds_kernel(int64_t t_first, int64_t t_last, int64_t *out)
{
    out[0] = t_first;
    out[1] = t_last;
}

// shared-memory budget of the per-window scheduler
static uint32_t smem_max_events()
{
    static uint32_t cached = 0;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (cached) return cached;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    uint64_t budget = (uint64_t)optin - 1024;  // static shared memory of the kernel
    uint32_t E = 64;
    while (arena_words(E + 64) * 4 <= budget) E += 64;
    cached = E;
    return cached;
}

template <typename T>
static cudaError_t alloc_async(T **p, uint64_t count, cudaStream_t st)
{
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    return cudaMallocAsync((void **)p, count * sizeof(T), st);
}

}  // namespace tn

using namespace tn;

// wait_end: return only once the plan's device buffers are written (else they
// are written by work enqueued on `stream`, which later users must follow)
static tn_status plan_create_impl(const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t m, uint32_t n,
                                  const int64_t *t_after, const tn_plan_options *opt, void *stream,
                                  tn_plan **plan_out, bool wait_end)
{
    if (!plan_out) return TN_EINVAL;
    *plan_out = nullptr;
    if (!u || !v || !t || m == 0 || n == 0 || n >= (1u << 30) || m >= (1ull << 30)) return TN_EINVAL;
    uint32_t sw = kDefaultSlab, window = kDefaultWindow, rows = 0, wave = 0, resident = 0;
    if (opt) {
        for (int i = 0; i < 2; ++i)
            if (opt->reserved[i]) return TN_EINVAL;
        if (opt->directed > 1) return TN_EINVAL;
        if (opt->slab_words) sw = opt->slab_words;
        if (opt->window_events) window = opt->window_events;
        rows = opt->smem_rows;
        wave = opt->wave_ctas;
        resident = opt->resident_words;
    }
    if (sw < 2 || sw > kMaxSlabWords || (sw & 1u)) return TN_EINVAL;  // even: whole 16-byte chunks
    if (window < 32) window = 32;
    if (resident) {
        // the resident-slab form keeps every row in shared memory: no row
        // buffer, and every window becomes level-ordered tiles of node-id ops
        // (a one-slot buffer holds no window that has an op)
        if ((resident != 1 && resident != 2) || opt->slab_words || opt->smem_rows || wave)
            return TN_EINVAL;
        if (n > resident_max_rows(resident)) return TN_EINVAL;
        rows = 1;
    }
    if (rows == 0) rows = (sw <= 16 ? kRowBufferBytes : kRowBufferWide) / (sw * 8);
    if (rows > kLocalSlotLimit) rows = kLocalSlotLimit;
    if ((uint64_t)rows * sw * 8 > kRowBufferWide) return TN_EINVAL;  // row buffer must fit the kernel's shared memory
    cudaStream_t st = (cudaStream_t)stream;
    tn_internal_keep_pool();

    PlanArgs a;
    memset(&a, 0, sizeof(a));
    a.u = u;
    a.v = v;
    a.t = t;
    a.m = m;
    a.n = n;
    a.t_after = t_after;
    a.window = window;
    a.directed = opt ? opt->directed : 0u;
    a.nw = (uint32_t)((m + window - 1) / window);
    a.smem_max_events = smem_max_events();
    a.dcap = rows;
    a.max_rec_words = kStageBytes / 4;

    tn_plan *p = (tn_plan *)calloc(1, sizeof(tn_plan));
    if (!p) return TN_ENOMEM;
    cudaGetDevice(&p->device);
    p->m = m;
    p->n = n;
    p->windows = a.nw;
    p->slab_words = sw;
    p->wave_ctas = wave;
    p->dcap = rows;
    p->resident = resident;

    tn_status rc = TN_OK;
    unsigned long long host_counters[4] = {0, 0, 0, 0};
    Totals host_tot;
    memset(&host_tot, 0, sizeof(host_tot));
    uint64_t *base = nullptr;
    Totals *d_tot = nullptr;
    const int vblocks = (int)((m + 255) / 256 < 4096 ? (m + 255) / 256 : 4096);
    const int wblocks = (int)((a.nw + 256) / 256);
    cudaError_t err = cudaSuccess;

#define TN_STEP(expr)                  \
    do {                               \
        err = (expr);                  \
        if (err != cudaSuccess) goto fail; \
    } while (0)

    TN_STEP(alloc_async(&a.counters, 4, st));
    TN_STEP(alloc_async(&a.wstart, (uint64_t)a.nw + 1, st));
    TN_STEP(alloc_async(&a.wcount, (uint64_t)kWinFields * a.nw, st));
    TN_STEP(alloc_async(&a.big_list, (uint64_t)a.nw, st));
    TN_STEP(alloc_async(&a.big_off, (uint64_t)a.nw, st));
    TN_STEP(cudaMemsetAsync(a.counters, 0, 4 * sizeof(unsigned long long), st));
    tn_internal_count_launches(3);
    validate_kernel<<<vblocks, 256, 0, st>>>(a);
    window_kernel<<<wblocks, 256, 0, st>>>(a);
    big_window_kernel<<<wblocks, 256, 0, st>>>(a);
    TN_STEP(cudaGetLastError());
    TN_STEP(cudaMemcpyAsync(host_counters, a.counters, sizeof(host_counters), cudaMemcpyDeviceToHost, st));
    // the batch's time bounds travel with the first synchronisation
    TN_STEP(cudaMemcpyAsync(&p->t_first, t, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    TN_STEP(cudaMemcpyAsync(&p->t_last, t + (m - 1), sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    TN_STEP(tn_internal_stream_wait(st));
    if (host_counters[0] & 1ull) {
        rc = TN_ERANGE;
        goto done;
    }
    if (host_counters[0] & 2ull) {
        rc = TN_EORDER;
        goto done;
    }
    p->big_windows = host_counters[1];

    TN_STEP(alloc_async(&a.ops_stage, 3 * m, st));
    TN_STEP(alloc_async(&a.aux_stage, 3 * m, st));
    TN_STEP(alloc_async(&a.lvl_stage, 2 * m + a.nw + 1, st));
    TN_STEP(alloc_async(&a.rec_stage, 10 * m + 8ull * a.nw, st));
    TN_STEP(alloc_async(&a.big_arena, host_counters[2], st));
    {
        const size_t smem = arena_words(host_counters[3] ? host_counters[3] : 1) * 4;
        TN_STEP(tn_internal_allow_max_dyn_smem((const void *)schedule_smem_kernel));
        tn_internal_count_launches(1);
        schedule_smem_kernel<<<a.nw, kPlanThreads, smem, st>>>(a);
        if (host_counters[1]) {
            tn_internal_count_launches(1);
            schedule_big_kernel<<<(unsigned)host_counters[1], kPlanThreads, 0, st>>>(a);
        }
        TN_STEP(cudaGetLastError());
    }
    TN_STEP(alloc_async(&base, 3ull * a.nw, st));
    TN_STEP(alloc_async(&d_tot, 1, st));
    tn_internal_count_launches(1);
    // 256 threads: the single scan CTA then fits an SM beside a running streaming
    // CTA (registers), instead of waiting for a free SM
    window_scan_kernel<<<1, 256, 0, st>>>(a.wcount, a.nw, base, d_tot);
    TN_STEP(cudaGetLastError());
    TN_STEP(cudaMemcpyAsync(&host_tot, d_tot, sizeof(Totals), cudaMemcpyDeviceToHost, st));
    TN_STEP(tn_internal_stream_wait(st));

    p->items = host_tot.items;
    p->blob8 = host_tot.blob8;
    p->aux = host_tot.naux;
    p->temps = host_tot.tmax;
    p->levels = host_tot.levels;
    p->ops = host_tot.ops;
    p->local_windows = host_tot.local;
    if (resident && !resident_fits(n, p->temps, resident)) {  // saved rows of the tie groups do not fit
        rc = TN_EINVAL;
        goto done;
    }
    TN_STEP(alloc_async(&p->d_blob, p->blob8 + 2, st));  // a global tile may read one op past its end
    TN_STEP(alloc_async(&p->d_items, p->items > 0 ? p->items : 1, st));
    TN_STEP(alloc_async(&p->d_aux, p->aux > 0 ? p->aux : 1, st));
    TN_STEP(alloc_async(&p->d_tbounds, 2, st));
    TN_STEP(alloc_async(&p->d_status, 1, st));
    TN_STEP(cudaMemsetAsync(p->d_status, 0, sizeof(int32_t), st));
    tn_internal_count_launches(2);
    compact_kernel<<<a.nw, 256, 0, st>>>(a, base, p->d_blob, p->d_items, p->d_aux);
    tbounds_kernel<<<1, 1, 0, st>>>(p->t_first, p->t_last, p->d_tbounds);
    TN_STEP(cudaGetLastError());
    // the plan is complete when this call returns, for use on any stream
    if (wait_end) TN_STEP(tn_internal_stream_wait(st));
    goto done;

fail:
    tn_internal_set_cuda_error(err);
    rc = err == cudaErrorMemoryAllocation ? TN_ENOMEM : TN_ECUDA;
done:
    cudaFreeAsync(a.counters, st);
    cudaFreeAsync(a.wstart, st);
    cudaFreeAsync(a.wcount, st);
    cudaFreeAsync(a.big_list, st);
    cudaFreeAsync(a.big_off, st);
    if (a.ops_stage) cudaFreeAsync(a.ops_stage, st);
    if (a.aux_stage) cudaFreeAsync(a.aux_stage, st);
    if (a.lvl_stage) cudaFreeAsync(a.lvl_stage, st);
    if (a.rec_stage) cudaFreeAsync(a.rec_stage, st);
    if (a.big_arena) cudaFreeAsync(a.big_arena, st);
    if (base) cudaFreeAsync(base, st);
    if (d_tot) cudaFreeAsync(d_tot, st);
    if (rc != TN_OK) {
        if (p->d_blob) cudaFreeAsync(p->d_blob, st);
        if (p->d_items) cudaFreeAsync(p->d_items, st);
        if (p->d_aux) cudaFreeAsync(p->d_aux, st);
        if (p->d_tbounds) cudaFreeAsync(p->d_tbounds, st);
        if (p->d_status) cudaFreeAsync(p->d_status, st);
        free(p);
        return rc;
    }
    *plan_out = p;
    return TN_OK;
#undef TN_STEP
}

extern "C" tn_status tn_plan_create(const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t m,
                                    uint32_t n, const int64_t *t_after, const tn_plan_options *opt,
                                    void *stream, tn_plan **plan_out)
{
    return plan_create_impl(u, v, t, m, n, t_after, opt, stream, plan_out, true);
}

tn_status tn::plan_create_ordered(const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t m, uint32_t n,
                                  const tn_plan_options *opt, cudaStream_t stream, tn_plan **plan_out)
{
    return plan_create_impl(u, v, t, m, n, nullptr, opt, stream, plan_out, false);
}

extern "C" tn_status tn_plan_destroy(tn_plan *p, void *stream)
{
    if (!p) return TN_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    cudaFreeAsync(p->d_blob, st);
    cudaFreeAsync(p->d_items, st);
    cudaFreeAsync(p->d_aux, st);
    cudaFreeAsync(p->d_tbounds, st);
    if (!p->status_shared) cudaFreeAsync(p->d_status, st);
    free(p);
    return TN_OK;
}

tn_status tn::plan_use_status(tn_plan *p, int32_t *status, cudaStream_t st)
{
    if (!p || !status) return TN_EINVAL;
    if (!p->status_shared) TN_CUDA_TRY(cudaFreeAsync(p->d_status, st));
    p->d_status = status;
    p->status_shared = 1;
    return TN_OK;
}

extern "C" tn_status tn_plan_get_stats(const tn_plan *p, tn_plan_stats *s)
{
    if (!p || !s) return TN_EINVAL;
    memset(s, 0, sizeof(*s));
    s->events = p->m;
    s->windows = p->windows;
    s->levels = p->levels;
    s->ops = p->ops;
    s->aux = p->aux;
    s->temps = p->temps;
    s->big_windows = p->big_windows;
    s->local_windows = p->local_windows;
    s->items = p->items;
    s->t_first = p->t_first;
    s->t_last = p->t_last;
    return TN_OK;
}

extern "C" tn_status tn_plan_status(tn_plan *p, void *stream)
{
    if (!p) return TN_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t h = 0;
    TN_CUDA_TRY(cudaMemcpyAsync(&h, p->d_status, sizeof(h), cudaMemcpyDeviceToHost, st));
    TN_CUDA_TRY(cudaMemsetAsync(p->d_status, 0, sizeof(int32_t), st));
    TN_CUDA_TRY(tn_internal_stream_wait(st));
    return (tn_status)h;
}
