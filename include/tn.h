/*
 * tn.h -- C ABI of the GB300 temporal out-component library (libtn).
 *
 * Method: "Temporal network compression via network hashing" (arXiv
 * 2307.04890).  A temporal network is a time-ordered list of undirected events
 * e = (u, v, t) between nodes u, v in [0, n) (Section 2.1).  Two events are
 * adjacent when they share a node and their times differ (dt > 0); node i is
 * reachable from node j when a time-respecting path of adjacent events leads
 * from j to i.  The component matrix S (Section 3.1) is the n x n boolean
 * matrix with S(i, j) = 1 iff i is reachable from j (or i == j): row i is the
 * in-component of i, column j the out-component of j.  Algorithm 1 builds it in
 * one pass: S <- I, then for every event r = S[u] | S[v]; S[u] = r; S[v] = r.
 * Events sharing a timestamp are applied as one snapshot (they do not chain):
 * S_new[x] = S_old[x] | OR over events (x, y) of the group of S_old[y].
 *
 * Network hashing (Section 4): R independent hash functions h_j map nodes to k
 * super-nodes; each maps the event stream to a proxy stream (h_j(u), h_j(v), t)
 * whose k x k component matrix P_j is computed with the same algorithm, and the
 * out-component of u is estimated by the intersection over j of the preimages
 * of OC_j(h_j(u)) (Section 4.2, eq. DefEstOCMerge).
 *
 * ---------------------------------------------------------------------------
 * Layout of a component matrix (all entry points)
 *   A matrix with `n_rows` rows and `ncols` source columns is stored row-major
 *   as uint64 words.  Each row occupies tn_row_words(ncols) words (a multiple of
 *   16 words = 128 bytes, so rows are 128-byte aligned); bit c of row i is
 *       (S[i * tn_row_words(ncols) + c / 64] >> (c % 64)) & 1
 *   and means "node i has been reached from source column c".  Bits at column
 *   positions >= ncols are zero on output.  For the full matrix ncols = n and
 *   column c is source node c.
 *
 * Pointers
 *   Unless a parameter says "host", every pointer is a DEVICE pointer on the
 *   current CUDA device, owned by the caller, and every call is enqueued on
 *   `stream` (a cudaStream_t; NULL = the legacy default stream).  The library
 *   keeps no reference to caller memory after a call returns, except that work
 *   it enqueued may still be reading or writing it until the stream reaches
 *   that point.  Scratch memory the library needs is taken from the CUDA
 *   stream-ordered allocator on `stream` and released on the same stream.
 *
 * Errors
 *   Every entry point returns a tn_status.  Host-detectable argument errors
 *   (NULL pointers, zero sizes where not allowed, sizes beyond the limits
 *   below) return TN_EINVAL before anything is enqueued.  Input checks that
 *   need the data (endpoint range, time order) run on the device and are
 *   returned synchronously by the calls documented as "validating" (they wait
 *   for their own small validation kernel).  Errors raised later inside
 *   asynchronous kernels (batch-order violations at apply time, bounded-wait
 *   timeouts) are recorded in a plan status word: read them with
 *   tn_plan_status().  No kernel of this library traps or asserts; a kernel
 *   that hits an error condition records it and returns.
 *
 * Limits: n < 2^30 nodes; m < 2^30 events per call or plan; k < 2^30.
 * Thread safety: calls on different plans and streams may run concurrently.
 */
#ifndef TN_H
#define TN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t tn_status;

#define TN_OK 0
#define TN_EINVAL (-1)   /* NULL pointer, zero or out-of-limit size, bad flag */
#define TN_ERANGE (-2)   /* an endpoint or a source id >= n */
#define TN_EORDER (-3)   /* timestamps decrease, or a batch does not start after t_last */
#define TN_ENOMEM (-4)   /* device scratch allocation failed */
#define TN_ECUDA (-5)    /* a CUDA runtime call failed */
#define TN_ETIMEOUT (-6) /* a bounded device-side wait expired */
#define TN_ESCRATCH (-7) /* the problem needs more than the fixed scratch of a no-alloc entry point */

/* Flags of tn_component_matrix / tn_component_columns / tn_plan_apply. */
#define TN_INIT_IDENTITY 1u /* initialise S first: identity, or the source columns */
#define TN_DIRECTED 4u      /* tn_component_matrix / tn_component_columns only: events
                               are directed u -> v (see tn_plan_options.directed) */
#define TN_REVERSE 2u       /* tn_component_matrix / tn_component_columns only: process
                               the sequence from its last timestamp group to its first
                               (Section 3.4); row i then ends as the OUT-component of i,
                               i.e. the result is the transpose of the chronological
                               matrix (with TN_DIRECTED the events are also turned
                               around, v -> u, so this still holds).  Requires
                               TN_INIT_IDENTITY and t_last == NULL
                               (it is not a streaming mode).  Scratch: 16 bytes per event. */

#define TN_GROUP_END 8u       /* tn_online_push only: the batch's last timestamp group is
                               complete (no later batch continues it) */

/* Human-readable name of a status code (static storage, never NULL). */
const char *tn_status_string(tn_status status);

/* Text of the last CUDA runtime error behind a TN_ECUDA / TN_ENOMEM returned
 * on the calling thread (diagnostics; static storage). */
const char *tn_last_cuda_error(void);

/* Row stride, in uint64 words, of a matrix with `ncols` source columns:
 * ceil(ncols / 1024) * 16 (rows padded to 128 bytes).  tn_row_words(0) = 0. */
uint64_t tn_row_words(uint64_t ncols);

/* ---------------------------------------------------------------------------
 * tn_component_matrix -- Algorithm 1 (Section 3.1) over one batch of events.
 *
 *   u, v   uint32[m] endpoints, each < n.
 *   t      int64[m] timestamps, non-decreasing (equal values form one
 *          snapshot group, Section 2.1: dt > 0 for adjacency).
 *   m      number of events; m == 0 is allowed (only the init, if flagged).
 *   n      number of nodes (rows and source columns).
 *   S      uint64[n * tn_row_words(n)], in/out.  With TN_INIT_IDENTITY it is
 *          first set to I_n; without it, S must hold the state reached by the
 *          earlier batches (streaming, Section 3.5: one pass, new events
 *          applied with the same rule).
 *   t_last int64 scalar, in/out, may be NULL.  When given, the batch must
 *          start strictly after *t_last (so no timestamp group is split across
 *          batches) and *t_last is set to t[m-1] when the batch is applied.
 *   flags  TN_INIT_IDENTITY or 0.
 * Validating: returns TN_ERANGE / TN_EORDER synchronously (S untouched).
 * The matrix update itself completes asynchronously on `stream`.
 */
tn_status tn_component_matrix(const uint32_t *u, const uint32_t *v, const int64_t *t,
                              uint64_t m, uint32_t n, uint64_t *S, int64_t *t_last,
                              uint32_t flags, void *stream);

/* ---------------------------------------------------------------------------
 * tn_init_matrix -- the initial state of Algorithm 1 (S <- I_n, Section 3.1).
 *
 *   S      uint64[n_rows * tn_row_words(ncols)] out.
 *   src    NULL: identity (ncols must equal n_rows); else uint32[ncols] source
 *          ids (< n_rows): bit c of row src[c] is set, everything else cleared.
 * Asynchronous without src; with src it is validating (an id >= n_rows
 * returns TN_ERANGE before anything is written).  Equivalent to the TN_INIT_IDENTITY step of
 * the calls below.
 */
tn_status tn_init_matrix(uint64_t *S, uint32_t n_rows, uint32_t ncols, const uint32_t *src,
                         void *stream);

/* Number of CUDA kernels this library has launched in the calling process
 * (all threads, all devices); for accounting in benchmarks and tests. */
uint64_t tn_kernel_launches(void);

/* ---------------------------------------------------------------------------
 * tn_component_columns -- the same algorithm restricted to the out-components
 * of the listed sources (columns of the component matrix are independent, so
 * any subset can be computed exactly on its own; Section 3.1).
 *
 *   src    uint32[nsrc] source node ids (< n, repeats allowed; an id >= n
 *          returns TN_ERANGE); column c of S is the out-component of src[c].
 *   S      uint64[n * tn_row_words(nsrc)], in/out; TN_INIT_IDENTITY sets bit c
 *          of row src[c] and clears everything else.
 * Other arguments and errors as tn_component_matrix.
 */
tn_status tn_component_columns(const uint32_t *u, const uint32_t *v, const int64_t *t,
                               uint64_t m, uint32_t n, const uint32_t *src, uint32_t nsrc,
                               uint64_t *S, int64_t *t_last, uint32_t flags, void *stream);

/* ---------------------------------------------------------------------------
 * tn_out_sizes -- component sizes (Section 3.1: out-component size = number
 * of ones in a column; Section 3.3, eq. for s_t: row and column sums have the
 * same total).
 *
 *   S          uint64[n_rows * tn_row_words(ncols)], as produced above.
 *   out_sizes  uint32[ncols] (required): out_sizes[c] = ones in column c.
 *   in_sizes   uint32[n_rows] or NULL: in_sizes[i] = ones in row i.
 *   argmax     uint32 scalar or NULL: the lowest column index holding the
 *              largest out-component.
 * Asynchronous; no device-side error conditions.
 */
tn_status tn_out_sizes(const uint64_t *S, uint32_t n_rows, uint32_t ncols,
                       uint32_t *out_sizes, uint32_t *in_sizes, uint32_t *argmax,
                       void *stream);

/* ---------------------------------------------------------------------------
 * Plans: the validated, scheduled form of one event batch.  tn_plan_create
 * checks the batch and builds its schedule once; tn_plan_apply then streams it
 * into any matrix over the same n (identity or source columns), as often as
 * needed, and contains no host synchronisation, so it can be captured in a
 * CUDA graph.  The plan owns its device memory.
 * ------------------------------------------------------------------------- */
typedef struct tn_plan tn_plan;

typedef struct tn_plan_options {
    uint32_t window_events; /* target events per scheduling window (0 = default 640) */
    uint32_t slab_words;    /* 64-bit words of every row owned by one CTA when the
                               plan is applied: an even number from 2 to 128
                               (0 = default 16).  Wide slabs (256-1024 byte row
                               segments) suit large networks whose windows stream
                               from global memory: fewer, longer DRAM bursts */
    uint32_t smem_rows;     /* row slots of the streaming kernel's shared-memory row
                               buffer (at most 192 KB / (8 slab_words)); windows with
                               more rows (plus saved copies) stream from global
                               memory (0 = 160 KB / (8 slab_words) for slabs of up to
                               16 words, 192 KB / (8 slab_words) above).  A buffer small
                               enough for two CTAs per SM (about 80 KB) runs two CTAs
                               of 4 consumer warps per SM; a larger one runs one CTA
                               of 12 consumer warps */
    uint32_t directed;      /* 1: event (u, v, t) is directed u -> v and only S[v] is
                               updated, S[v] |= S[u] (the paper's footnote to Section
                               3.1); timestamp groups stay snapshots.  0: undirected */
    uint32_t wave_ctas;     /* 0: one CTA per slab_words-wide slab, ceil(row words /
                               slab_words) CTAs per matrix.  N > 0: the row is
                               spread over N CTAs of at most slab_words words each
                               (two widths that differ by one unit; the unit is
                               16 words, 128 bytes, when slab_words is a multiple
                               of 16 and the row has at least N such units, else
                               2 words), e.g. one full wave of the GPU's SMs.  N
                               below ceil(row words / slab_words) is raised to it */
    uint32_t resident_words;/* 0: the column-slab form above (rows move between HBM and
                               shared memory).  1 or 2: the resident-slab form for
                               small networks, the same update of Algorithm 1
                               (Section 3.1) in another launch shape: each CTA keeps
                               resident_words 64-bit
                               words of EVERY row (and of the tie groups' saved rows)
                               in shared memory for the whole batch and reads only the
                               schedule, so the matrix is read and written once per
                               application.  Needs (n + saved rows) * 8 *
                               resident_words bytes of shared memory per CTA:
                               tn_plan_create returns TN_EINVAL when n is above
                               tn_resident_max_rows(resident_words) or the tie groups'
                               saved rows do not fit beside the rows.  slab_words,
                               smem_rows and wave_ctas must then be 0.  The plan
                               applies like any other (identity, source columns,
                               t_last, batches and graphs, mixed with column-slab
                               plans in one launch); tn_online_create rejects it */
    uint32_t reserved[2];   /* must be zero */
} tn_plan_options;

/* A launch-shape helper with no counterpart in the paper: the largest node
 * count n whose rows fit the resident-slab form at
 * `resident_words` (1 or 2) 64-bit words per row, with no saved rows (a
 * plan whose tie groups need saved rows needs room for them too): 24,928 and
 * 12,464 on a GB300.  0 for an unsupported width, or when the current device
 * cannot be queried.  No device work: the first call per device queries its
 * shared-memory limit. */
uint32_t tn_resident_max_rows(uint32_t resident_words);

typedef struct tn_plan_stats {
    uint64_t events;     /* m */
    uint64_t windows;    /* scheduling windows */
    uint64_t levels;     /* dependency levels (barriers per applied slab) */
    uint64_t ops;        /* row operations after tie handling */
    uint64_t aux;        /* source-list entries of multi-source updates */
    uint64_t temps;      /* saved-row slots needed by tie groups (max per window) */
    uint64_t big_windows;  /* windows scheduled by the large-window path */
    uint64_t local_windows;/* windows applied in shared memory */
    uint64_t items;        /* work items of the streaming kernel */
    int64_t t_first, t_last;
} tn_plan_stats;

/* Validating.  u, v, t, m, n as tn_component_matrix (m >= 1).
 * t_after: device int64 scalar or NULL; when given the batch must satisfy
 * t[0] > *t_after (TN_EORDER otherwise).  opt may be NULL.  On success *plan
 * receives a new plan.  The caller may free u, v, t once this call returns. */
tn_status tn_plan_create(const uint32_t *u, const uint32_t *v, const int64_t *t,
                         uint64_t m, uint32_t n, const int64_t *t_after,
                         const tn_plan_options *opt, void *stream, tn_plan **plan);

/* Streams the plan's events into S (layout above, ncols columns).
 *   src    NULL for the full matrix (ncols must equal n), or uint32[ncols]
 *          source ids for a column subset (used only with TN_INIT_IDENTITY).
 *   t_last device int64 scalar or NULL: checked on the device
 *          (plan t_first > *t_last, else the plan status becomes TN_EORDER and
 *          S is left untouched) and then set to the plan's t_last.
 * Asynchronous. */
tn_status tn_plan_apply(const tn_plan *plan, uint64_t *S, uint32_t ncols,
                        const uint32_t *src, int64_t *t_last, uint32_t flags,
                        void *stream);

/* One launch over several (plan, matrix) pairs (networks of different n and
 * m, e.g. the R proxies of a hashed network, together with the sampled exact
 * columns of the network they stand for): count entries of each array.
 * src may be NULL (every matrix has one column per node) or hold count
 * entries, each NULL or the device source-id list of that matrix's ncols
 * columns, as in tn_plan_apply (used only with TN_INIT_IDENTITY; ids >= n are
 * recorded as TN_ERANGE in that plan's status).  Equivalent to calling
 * tn_plan_apply on each pair; all pairs must use distinct S buffers.
 * Asynchronous, capturable. */
tn_status tn_plan_apply_batch(const tn_plan *const *plans, uint64_t *const *S,
                              const uint32_t *ncols, const uint32_t *const *src,
                              uint32_t count, uint32_t flags, void *stream);

/* Waits for `stream`, then returns and clears the first error recorded by an
 * asynchronous kernel that used this plan (TN_OK if none). */
tn_status tn_plan_status(tn_plan *plan, void *stream);

tn_status tn_plan_get_stats(const tn_plan *plan, tn_plan_stats *stats);

/* Releases the plan; its memory is returned on `stream` after the work
 * already enqueued there. */
tn_status tn_plan_destroy(tn_plan *plan, void *stream);

/* ---------------------------------------------------------------------------
 * Batched application as a CUDA graph (Section 4.2: the R proxy networks of a
 * hashed network are independent and are built together).
 *
 * tn_graph_capture_batch records one tn_plan_apply_batch of these arguments
 * (with `flags`) into a CUDA graph on a private stream and instantiates it;
 * tn_graph_launch replays it on `stream` (one launch), recomputing the same
 * matrices from the same plans.  The plans and matrices must stay alive and
 * unchanged in size while the graph exists.  The first plan status error
 * still gates the replay as it gates a direct call.
 */
typedef struct tn_graph tn_graph;

tn_status tn_graph_capture_batch(const tn_plan *const *plans, uint64_t *const *S,
                                 const uint32_t *ncols, uint32_t count, uint32_t flags,
                                 tn_graph **graph);
tn_status tn_graph_launch(tn_graph *graph, void *stream);
tn_status tn_graph_destroy(tn_graph *graph);

/* ---------------------------------------------------------------------------
 * tn_autotune -- picks the plan options (slab width = columns per CTA, window
 * depth, shared-memory row buffer = CTAs per SM) for a batch of `replicas`
 * networks shaped like (u, v, t, m, n), each with `ncols` source columns
 * (0 = n; fewer = a column subset as in tn_component_columns).  The full problem runs replicas x
 * ceil(row words / slab) CTAs in waves of (SMs x CTAs per SM); every candidate
 * is timed on the first `sample_events` events (0 = all) over one wave's worth
 * of CTAs -- whole scratch matrices for small n, the first source columns for
 * large n (columns are independent) -- and scored as waves x that time plus
 * replicas x the time tn_plan_create takes on the sample.
 * Candidates of the column-slab form: slab 2/4/8/12/16/24/32/48/64 words (at
 * most the row width), window 320/640/1024 events, row buffer 160 or 80 KB
 * (192 KB above 16 words).  Candidates of the resident-slab form, when the
 * network's rows fit (tn_resident_max_rows): resident_words 1/2, window
 * 640/2048 events.  Scratch of one timing run is kept under half of the free
 * device memory and 64 GiB.  The choice is cached per (device, n, ncols,
 * replicas, floor(log2 m)) for the life of the process.  Synchronous.
 */
typedef struct tn_tune_result {
    tn_plan_options best;   /* options to pass to tn_plan_create */
    float best_ms;          /* its score: waves x timed sample + replicas x plan time (ms) */
    uint32_t tried;         /* candidates timed */
    uint32_t cached;        /* 1 if the result came from the cache */
    uint32_t pad;
    uint64_t sample_events;
} tn_tune_result;

tn_status tn_autotune(const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t m,
                      uint32_t n, uint32_t ncols, uint32_t replicas, uint64_t sample_events,
                      void *stream, tn_tune_result *result);

/* ---------------------------------------------------------------------------
 * tn_hash_proxy -- network hashing (Section 4.1).
 *
 * Hash family: Thorup-Zhang 2-character tabulation with a derived character.
 * For replica j < R the coefficients A(i, c), i < 3, c < 4, are
 * ((r1 << 32) + r2) mod (2^61 - 1) where r1, r2, ... is a SplitMix64 stream
 * (Steele, Lea, Flood 2014) started at state splitmix64(seed XOR j) and each
 * draw is reduced modulo 2^31 - 1; draws go in the order i, c, r1, r2.
 * T_i[x] = A(i,0) x^3 + A(i,1) x^2 + A(i,2) x + A(i,3) mod 2^61 - 1 (Horner),
 * and h_j(u) = (T0[u & 0xFFFF] ^ T1[u >> 16] ^ T2[(u & 0xFFFF) + (u >> 16)]) mod k.
 *
 *   H      uint32[R * n] out: H[j * n + x] = h_j(x).
 *   pu, pv uint32[R * m] out, may both be NULL: the super-events of replica j
 *          are (pu[j*m + e], pv[j*m + e], t[e]); the timestamps are unchanged.
 *   u, v   uint32[m] endpoints (< n); may be NULL when m == 0.
 * Asynchronous.  Endpoints >= n are not hashed: their super-events get the
 * invalid id 0xFFFFFFFF, which a later plan over them rejects (TN_ERANGE).
 */
tn_status tn_hash_proxy(const uint32_t *u, const uint32_t *v, uint64_t m, uint32_t n,
                        uint32_t k, uint32_t R, uint64_t seed, uint32_t *H,
                        uint32_t *pu, uint32_t *pv, void *stream);

/* ---------------------------------------------------------------------------
 * tn_hash_estimate -- fusion (Section 4.2, eqs. DefInvHComp, DefEstOCMerge):
 *   est[s] = #{ w in [0, n) : for all j < R, bit h_j(x) of row h_j(w) of P_j }
 * with x = src[s] (or x = s when src is NULL and nsrc == n).
 *
 *   P    uint64[R * k * tn_row_words(k)]: the R proxy component matrices,
 *        each k x k in the layout above, stored one after the other.
 *   H    uint32[R * n] as written by tn_hash_proxy.
 *   est  uint32[nsrc] out.
 * Asynchronous when src is NULL; validating with src (ids >= n: TN_ERANGE).
 */
tn_status tn_hash_estimate(const uint64_t *P, uint32_t R, uint32_t k, const uint32_t *H,
                           uint32_t n, const uint32_t *src, uint32_t nsrc, uint32_t *est,
                           void *stream);

/* ---------------------------------------------------------------------------
 * tn_error_stats -- error of estimated against exact out-component sizes of
 * the same sources (Section 4.4 reports the Earth-Mover distance between the
 * estimated and the exact size distributions).
 *
 *   est, exact  uint32[count] (device): est[s] and exact[s] belong to the same
 *               source; every exact size is >= 1 (a node reaches itself).
 *   max_value   bound on every value (e.g. n); sizes the histograms.
 *   out         HOST pointer, filled on success:
 *     sum_abs  = sum |est - exact|          max_abs = max |est - exact|
 *     w1_num   = count * W1, W1 the Wasserstein-1 distance between the two
 *                empirical distributions = sum over integers x of
 *                |#{est <= x} - #{exact <= x}| / count (exact integers)
 *     rel_sum  = sum |est - exact| / exact  max_rel = max of the same (double;
 *                rel_sum is summed in an unspecified order)
 *     mean_abs = sum_abs / count, mean_rel = rel_sum / count, w1 = w1_num / count.
 * Synchronous (waits for `stream`).  TN_ERANGE if a value exceeds max_value or
 * an exact size is 0.  Scratch: 8 * (max_value + 1) bytes from the
 * stream-ordered allocator.
 */
typedef struct tn_error_stats {
    uint64_t count, sum_abs, max_abs, w1_num;
    double rel_sum, max_rel, mean_abs, mean_rel, w1;
} tn_error_stats;

tn_status tn_error_stats_compute(const uint32_t *est, const uint32_t *exact, uint32_t count,
                                 uint32_t max_value, tn_error_stats *out, void *stream);

/* ---------------------------------------------------------------------------
 * tn_hash_estimate_noalloc -- the same fusion as tn_hash_estimate (same
 * arguments, same result bit for bit, but always the byte-table form: one CTA
 * per 8 sources, each reading all of H, so its cost grows as ceil(nsrc / 8)
 * reads of H where tn_hash_estimate switches to bit-sliced tables at 256
 * sources) for callers that cannot allocate device
 * memory while they run: code that executes inside another framework's memory
 * pool or budget (where a cudaMalloc or a stream-ordered allocation would go
 * around the owner's accounting or fail once the budget is reserved), and
 * latency-bound loops where an allocation could synchronise the device or
 * stall.  The paper has no counterpart to this entry point: it only changes
 * where the scratch lives.
 *
 * It allocates nothing: no cudaMalloc / cudaFree / stream-ordered allocator or
 * allocating library call.  Its scratch is one fixed device array of
 * TN_NOALLOC_SCRATCH_BYTES bytes per device, owned by the library (static
 * storage of the library's module, held on every GPU that loads the library
 * until the process exits), whose address is looked up once per device on the
 * first call made with that device current:
 *   - a 4-byte flag for the source-id check, cleared on the stream before
 *     every validating call;
 *   - the per-CTA fusion tables when R * k exceeds the 200 KiB shared-memory
 *     table: R * k * ceil(nsrc / 8) bytes, at most TN_NOALLOC_TABLE_BYTES.
 *     A problem that needs more returns TN_ESCRATCH before anything is
 *     enqueued (use tn_hash_estimate, which allocates, or fewer sources).
 * The scratch is shared by every call on a device: calls that overlap in time
 * (other streams, other threads) race on it, so serialise them.  The first
 * call on a device resolves the scratch address and must come before any
 * stream capture; nothing is claimed about capturing this call in a graph.
 * Asynchronous when src is NULL; validating with src (ids >= n: TN_ERANGE).
 */
#define TN_NOALLOC_TABLE_BYTES (8u << 20)
#define TN_NOALLOC_SCRATCH_BYTES (TN_NOALLOC_TABLE_BYTES + 256u)
tn_status tn_hash_estimate_noalloc(const uint64_t *P, uint32_t R, uint32_t k, const uint32_t *H,
                                   uint32_t n, const uint32_t *src, uint32_t nsrc, uint32_t *est,
                                   void *stream);

/* ---------------------------------------------------------------------------
 * Serving (Section 3.5: the method is a one-pass streaming algorithm, so a
 * job's matrix can stay on the device while its event batches arrive).
 *
 * A server runs worker threads on the device that is current when it is
 * created.  A job is opened (tn_server_open: n nodes, a bound on the events of
 * any one of its batches, the host buffers of its results) and then receives
 * its event batches one at a time (tn_server_push), the last one flagged
 * TN_LAST_BATCH.  Jobs are admitted in open order whenever fewer than
 * max_active jobs are resident and the job's device memory (tn_server_job_bytes)
 * fits in memory_budget, so jobs that arrive while others run join the device
 * as soon as a slot and memory free up; batches pushed before admission wait
 * in the job.  An admitted job owns an online state (tn_online_*: S <- I, then
 * every batch in push order; a timestamp group split by a batch boundary is
 * held back until the group is complete, Section 2.1) on a stream of its own;
 * a worker copies each pushed batch in and pushes it to the job's state while
 * the job's earlier batches and other jobs run on the device.  After the last
 * batch the out-sizes (and the largest out-component) are copied to the
 * caller's host buffers.  Results are exactly those of
 * tn_out_component_sizes_host on the concatenated events.
 *
 * Each resident job uses two streams (scheduling, updates).  A process that
 * serves many jobs at once should raise CUDA_DEVICE_MAX_CONNECTIONS (an
 * environment variable read when the CUDA context is created) to 32: with the
 * default 8 hardware work queues, a job's short scheduling kernels queue behind
 * other jobs' long-running updates that share their hardware queue.
 */
typedef struct tn_server tn_server;

typedef struct tn_server_options {
    uint64_t memory_budget; /* device bytes for resident jobs (0 = 60 % of free memory) */
    uint32_t max_active;    /* jobs resident at once (0 = 16) */
    uint32_t window_events; /* plan options of every batch (0 = windows of 576 events and a
                               144 KB row buffer, which leave room on each SM for the
                               scheduling CTAs of other jobs' batches beside a running
                               update CTA; else this window and the default buffer) */
    uint32_t slab_words;    /* 0 = per job: the widest even slab (at most 16 words)
                               that still gives the job 16 CTAs, at least 2 words */
    uint32_t workers;       /* host worker threads (0 = 16): admission, copies in,
                               scheduling of batches */
    uint32_t reserved[2];   /* must be zero */
} tn_server_options;

typedef struct tn_job_record {
    uint64_t job_id;
    int32_t status;           /* TN_OK, or the job's error (e.g. TN_EORDER, TN_ERANGE) */
    uint32_t n;
    uint64_t events;
    uint64_t t_submit_ns;     /* host steady-clock times: open, */
    uint64_t t_admit_ns;      /* admission, */
    uint64_t t_done_ns;       /* results on the host, */
    uint64_t t_last_push_ns;  /* the push of the last batch, */
    uint64_t t_enqueued_ns;   /* and the end of the host work of the last batch
                                 (copied in, scheduled, results enqueued) */
} tn_job_record;

typedef struct tn_server_stats {
    uint64_t queued, active, admitted, completed;
    uint64_t bytes_in_use, budget, peak_active, peak_bytes;
    /* host time spent by the workers, summed over them (ns): admitting jobs
     * (streams, state, buffers), copying batches in, pushing them to the
     * jobs' online states (validation and scheduling, which wait for the
     * planner's kernels), enqueueing results, and retiring finished jobs */
    uint64_t batches;
    uint64_t admit_ns, copy_ns, schedule_ns, result_ns, retire_ns;
} tn_server_stats;

#define TN_LAST_BATCH 16u     /* tn_server_push: the job's last batch */

tn_status tn_server_create(const tn_server_options *opt, tn_server **server);

/* Device bytes charged to the memory budget for a job of n nodes whose
 * batches hold at most max_batch_events events: its matrix (rows rounded up
 * to a multiple of 1,024 as in the online state), sizes, and per batch being
 * scheduled 160 bytes per event (copy in, held-back group, schedule). */
uint64_t tn_server_job_bytes(uint32_t n, uint64_t max_batch_events);

/* Opens job `job_id` (unique among the server's open jobs): n nodes, batches of
 * at most max_batch_events events, out_sizes a HOST uint32[n], argmax a HOST
 * uint32 or NULL (both written when the job finishes).  TN_ENOMEM if the job
 * could never fit the budget, TN_EINVAL for a bad argument or a job id that
 * is already open. */
tn_status tn_server_open(tn_server *server, uint64_t job_id, uint32_t n, uint64_t max_batch_events,
                         uint32_t *out_sizes, uint32_t *argmax);

/* Appends a batch to an open job: HOST arrays u, v (uint32, < n) and t (int64,
 * non-decreasing, continuing the job's earlier batches; equal timestamps may
 * span a boundary) of m <= max_batch_events events, pinned or pageable, kept
 * alive by the caller until the job's record is returned by tn_server_poll.
 * flags: 0 or TN_LAST_BATCH (no further batches: the job's results follow).
 * A batch out of order or out of range ends the job with TN_EORDER /
 * TN_ERANGE in its record.  TN_EINVAL for an unknown or closed job. */
tn_status tn_server_push(tn_server *server, uint64_t job_id, const uint32_t *u, const uint32_t *v,
                         const int64_t *t, uint64_t m, uint32_t flags);

/* Open + one push per batch: HOST arrays u, v, t of batch_offsets[nbatches]
 * events, batch b = [batch_offsets[b], batch_offsets[b+1]) (batch_offsets[0] =
 * 0, non-decreasing, each batch < 2^30 events). */
tn_status tn_server_submit(tn_server *server, uint64_t job_id, uint32_t n, const uint32_t *u,
                           const uint32_t *v, const int64_t *t, const uint64_t *batch_offsets,
                           uint32_t nbatches, uint32_t *out_sizes, uint32_t *argmax);

/* Moves up to `capacity` records of finished jobs (in completion order) into
 * `records`; waits up to wait_ms for the first one.  *count = records moved. */
tn_status tn_server_poll(tn_server *server, tn_job_record *records, uint32_t capacity,
                         uint32_t *count, uint32_t wait_ms);

tn_status tn_server_get_stats(tn_server *server, tn_server_stats *stats);

/* Finishes every admitted and queued job whose last batch was pushed (a job
 * that never receives its last batch is dropped with its pending batches),
 * then stops the workers and frees the server (records not yet polled are
 * dropped). */
tn_status tn_server_destroy(tn_server *server);

/* ---------------------------------------------------------------------------
 * Node growth (Section 3.5, advantages and limitations of the matrix method:
 * a node that joins the network adds a row and a column to the component
 * matrix: zeros, except the new node's own diagonal bit).
 *
 * tn_grow_matrix -- S_new (n_new x n_new, layout above) receives S_old
 * (n_old x n_old) in its first n_old rows and columns, with bits of columns
 * >= n_old cleared, and the identity on the new nodes:
 *   S_new[i][j] = S_old[i][j] for i, j < n_old;  S_new[i][i] = 1 for i >= n_old;
 *   every other bit 0.
 *   S_old  uint64[n_old * tn_row_words(n_old)], may be NULL when n_old == 0.
 *   S_new  uint64[n_new * tn_row_words(n_new)]; either disjoint from S_old, or
 *          equal to it when tn_row_words(n_new) == tn_row_words(n_old) (in
 *          place: the buffer must already hold n_new rows; only the new rows
 *          and the new columns of the old rows are written).
 * TN_EINVAL for n_new < n_old, n_new >= 2^30, partially overlapping buffers,
 * an in-place call whose row stride would change, or a pointer that is not
 * 16-byte aligned.  Asynchronous.
 */
tn_status tn_grow_matrix(const uint64_t *S_old, uint32_t n_old, uint64_t *S_new, uint32_t n_new,
                         void *stream);

/* ---------------------------------------------------------------------------
 * Online state (Section 3.5: one pass over the events, new events and new
 * nodes processed as they arrive).  The object owns a component matrix on the
 * device that starts as I_n and takes event batches in time order and node
 * growth at any point between them.
 *
 * Timestamp groups may be split across batches.  A group is one snapshot
 * (Section 2.1: adjacency needs dt > 0), so none of its events may be applied
 * before all of them are known: every push holds back the events of the
 * batch's last timestamp ("pending") and applies them with the next batch,
 * whose first events may continue the same group, unless the push carries
 * TN_GROUP_END.  After a push, S therefore holds every pushed event with a
 * timestamp below the pending one; after tn_online_flush (or a push with
 * TN_GROUP_END) it holds all of them, and the next batch must start at a
 * strictly later timestamp.  The result equals tn_component_matrix over the
 * concatenation of the batches (on the grown matrix, where nodes were added).
 *
 * All calls of one object must come from one host thread at a time, on one
 * device (the one current at create); the matrix and the held-back events
 * live in the stream-ordered pool, and `stream` may differ between calls only
 * if the caller orders those streams.
 */
typedef struct tn_online tn_online;

typedef struct tn_online_state {
    uint64_t *S;             /* device matrix, n x row_words words; moves when a
                                tn_online_grow changes the row stride */
    uint32_t n;              /* current number of nodes */
    uint32_t has_applied;    /* 1 once any event has been applied to S */
    uint64_t row_words;      /* tn_row_words(n) */
    uint64_t pending_events; /* events held back (timestamp pending_t) */
    int64_t pending_t;
    int64_t t_applied;       /* last timestamp applied to S (if has_applied) */
    uint64_t applied_events; /* events applied to S so far */
    uint64_t batches;        /* pushes accepted */
} tn_online_state;

/* Creates the state for n nodes (S <- I_n, Algorithm 1).  opt as for
 * tn_plan_create (NULL = defaults; opt->directed selects directed events).
 * TN_EINVAL for n == 0, n >= 2^30 or bad options. */
tn_status tn_online_create(uint32_t n, const tn_plan_options *opt, void *stream, tn_online **online);

/* Pushes a batch: u, v uint32[m] (device, < current n), t int64[m] (device,
 * non-decreasing).  Its first timestamp must be >= the pending timestamp when
 * events are pending (equal: the batch continues the pending group), else
 * > the last applied timestamp.  flags: 0 or TN_GROUP_END.  m == 0 is allowed
 * (with TN_GROUP_END it applies the pending group).  Validating and
 * synchronous up to the scheduling of the complete groups (TN_ERANGE,
 * TN_EORDER leave the state unchanged); the matrix update runs on `stream`
 * after the call returns and may be read by later work on that stream.  A
 * device error of an applied batch is returned by the next call on the
 * object.  The caller may reuse u, v, t once the call returns. */
tn_status tn_online_push(tn_online *online, const uint32_t *u, const uint32_t *v, const int64_t *t,
                         uint64_t m, uint32_t flags, void *stream);

/* Applies the pending group (same as a push of no events with TN_GROUP_END). */
tn_status tn_online_flush(tn_online *online, void *stream);

/* Adds nodes n .. n_new - 1 (tn_grow_matrix on the owned matrix; in place
 * while the row stride stays, else into a new buffer).  Pending events stay
 * pending; later batches may use the new ids.  TN_EINVAL for n_new < n. */
tn_status tn_online_grow(tn_online *online, uint32_t n_new, void *stream);

/* Waits for `stream` and returns the first device error of an applied batch
 * (TN_OK if none); the error is sticky. */
tn_status tn_online_status(tn_online *online, void *stream);

/* Host-side snapshot of the state (no synchronisation). */
tn_status tn_online_get_state(const tn_online *online, tn_online_state *state);

/* Frees the object; its memory is returned on `stream` after the work already
 * enqueued there. */
tn_status tn_online_destroy(tn_online *online, void *stream);

/* ---------------------------------------------------------------------------
 * HyperLogLog sketches of the components (Section 3.3; with TN_REVERSE,
 * Section 3.4).  Approximate: O(n s)
 * memory instead of n^2 bits, for the average component size (in-components,
 * Eq. s_t) or, with TN_REVERSE, the out-component size distribution.
 *
 * Node i keeps s = 2^p one-byte registers (4 <= p <= 16).  Element x hashes to
 * h = one SplitMix64 step (Steele, Lea, Flood 2014) from state (seed XOR x);
 * its register is the top p bits of h, its rank the position of the first 1
 * among the remaining 64 - p bits (64 - p + 1 if none).  Node i starts as the
 * sketch of {i}; every event merges sketches by register-wise maximum under
 * the same rules as the component matrix (snapshot timestamp groups, flags
 * TN_REVERSE and TN_DIRECTED as for tn_component_matrix), so row i is exactly
 * the sketch of node i's in-component (out-component when reversed).
 *
 *   R    uint8, n rows of tn_hll_row_bytes(p) bytes (a multiple of 128),
 *        16-byte aligned; register j of node i is R[i * row_bytes + j].
 * Validating and synchronous (TN_ERANGE for an endpoint >= n).
 */
uint64_t tn_hll_row_bytes(uint32_t p);  /* 0 for p outside [4, 16] */
tn_status tn_hll_sketches(const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t m,
                          uint32_t n, uint32_t p, uint64_t seed, uint32_t flags, uint8_t *R,
                          void *stream);

/* est[i] = alpha_s s^2 / sum_j 2^(-M[j]) for node i's registers M (alpha_16
 * 0.673, alpha_32 0.697, alpha_64 0.709, else 0.7213 / (1 + 1.079 / s)),
 * replaced by linear counting s ln(s / V) when it is <= 2.5 s and V > 0
 * registers are zero (Flajolet et al. 2007).  est: double[n].  Asynchronous. */
tn_status tn_hll_estimate(const uint8_t *R, uint32_t n, uint32_t p, double *est, void *stream);

/* ---------------------------------------------------------------------------
 * tn_selftest_wait_timeout -- exercises the bounded device waits that every
 * kernel of this library uses instead of unbounded spins: a kernel waits on a
 * barrier that nothing completes and gives up after its poll limit (a few
 * seconds at most).  Returns TN_ETIMEOUT when the bounded wait works (the
 * context stays usable), TN_OK never.  Synchronous.  No counterpart in the
 * paper: it checks this library's failure handling.
 */
tn_status tn_selftest_wait_timeout(void *stream);

/* ---------------------------------------------------------------------------
 * tn_out_component_sizes_host -- the whole exact path from HOST arrays:
 * copies u, v, t (host, pinned or pageable) to the device, builds the
 * component matrix from the identity (Algorithm 1, Section 3.1), computes the
 * out-sizes (Section 3.3) and copies them back.  opt: plan options (window,
 * slab width, row buffer, wave spread, direction; NULL = defaults), as for
 * tn_plan_create.  out_sizes is a HOST uint32[n]; argmax a HOST uint32 or
 * NULL.  Synchronous: returns when the host outputs are written.  Device
 * memory is taken from and returned to the stream-ordered allocator.
 */
tn_status tn_out_component_sizes_host(const uint32_t *u, const uint32_t *v, const int64_t *t,
                                      uint64_t m, uint32_t n, const tn_plan_options *opt,
                                      uint32_t *out_sizes, uint32_t *argmax, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TN_H */
