/*
 * tnref -- CPU oracle for temporal out-components and network hashing.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the GPU library is checked against.  Only the test suite, the
 * package smoke check and the benchmark's CPU-baseline leg may load it; the
 * product path never does.  It shares no code, header or table with the GPU
 * library.
 *
 * Conventions (paper Section 2.1): an event e = (u, v, t) is an undirected
 * interaction between nodes u, v in [0, n) at integer time t; events arrive
 * sorted by non-decreasing t.  Two events are adjacent only when they share a
 * node AND their times differ (dt > 0), so events with equal timestamps never
 * chain.  A "component matrix" has n rows of `width` uint64 words (row stride =
 * width, no padding); bit c of row i is (S[i*width + c/64] >> (c%64)) & 1 and
 * means "node i has been reached from source column c" (Section 3.1: row i is
 * the in-component of i, column j the out-component of j).
 *
 * Readings of the paper that this file fixes (the paper is silent or garbled):
 *  - equal timestamps: a group G of events with the same t is applied as one
 *    snapshot, S_new[x] = S_old[x] OR (OR over e in G touching x of
 *    S_old[other end of e]).  With distinct timestamps this is exactly
 *    Algorithm 1 (one event at a time: r = S[u] | S[v]; S[u] = S[v] = r).
 *  - self-loops and duplicate events are harmless no-ops of the same rule.
 *  - the hash is Thorup-Zhang 2-character tabulation with derived character
 *    (Section 4.1), tables filled by degree-3 polynomials modulo 2^61-1 whose
 *    coefficients come from a SplitMix64 stream reduced modulo 2^31-1.
 *
 * Parity status: the component matrix, its sizes, the recombination and the
 * brute-force SI simulation are pinned by the tests (closed forms, brute force,
 * invariants).  The hash's exact constants are a project definition: the
 * SplitMix64 stream is pinned by the generator's known-answer values, the
 * coefficient rule and the tables by big-integer restatements, and the
 * structure and 4-wise independence by statistical tests.  Agreement with the
 * authors' own (unpublished) hash values cannot be checked.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TNREF_OK 0
#define TNREF_EINVAL (-1)
#define TNREF_ERANGE (-2)
#define TNREF_EORDER (-3)
#define TNREF_ENOMEM (-4)

/* ---------------------------------------------------------------------------
 * Input checks (Section 2.1: nodes are labelled [0, n), events are time
 * ordered).
 * ------------------------------------------------------------------------- */
int tnref_validate(const uint32_t *u, const uint32_t *v, const int64_t *t,
                   uint64_t m, uint32_t n)
{
    for (uint64_t e = 0; e < m; ++e) {
        if (u[e] >= n || v[e] >= n)
            return TNREF_ERANGE;
        if (e > 0 && t[e] < t[e - 1])
            return TNREF_EORDER;
    }
    return TNREF_OK;
}

/* ---------------------------------------------------------------------------
 * Initial state (Algorithm 1, first line: S <- I_n).  Column c of the matrix
 * is the out-component of source node src[c]; with src == NULL the sources are
 * all n nodes in order and the result is the identity matrix.  Columns not
 * covered by a source stay zero.
 * ------------------------------------------------------------------------- */
void tnref_init_sources(uint64_t *S, uint32_t n, uint64_t width,
                        const uint32_t *src, uint64_t nsrc)
{
    memset(S, 0, (size_t)n * width * sizeof(uint64_t));
    if (src == NULL) {
        for (uint32_t i = 0; i < n; ++i)
            S[(uint64_t)i * width + i / 64] |= 1ull << (i % 64);
    } else {
        for (uint64_t c = 0; c < nsrc; ++c)
            S[(uint64_t)src[c] * width + c / 64] |= 1ull << (c % 64);
    }
}

/* ---------------------------------------------------------------------------
 * The matrix algorithm (Algorithm 1, Section 3.1) with equal-timestamp groups
 * applied as snapshots (adjacency requires dt > 0, Section 2.1).
 *
 * For each group G of equal t, in time order:
 *   old[x] = S[x] for every node x touched by G;
 *   for each event (a, b) in G:  S[a] |= old[b];  S[b] |= old[a].
 * Because S[a] already contains old[a], a singleton group gives
 * S[a] = S[b] = old[a] | old[b], which is Algorithm 1's update.
 * ------------------------------------------------------------------------- */
/* One timestamp group [g0, g1) applied as a snapshot: every endpoint's row
 * gets the OR of its partners' rows as they were before the group. */
struct tnref_groups {
    int64_t *slot;
    uint32_t *touched;
    uint64_t *old;
    uint64_t cap;
};

static int apply_group(struct tnref_groups *gs, const uint32_t *u, const uint32_t *v, uint64_t g0,
                       uint64_t g1, uint64_t *S, uint64_t width)
{
    uint64_t need = 2 * (g1 - g0);
    if (need > gs->cap) {
        free(gs->touched);
        free(gs->old);
        gs->cap = need;
        gs->touched = (uint32_t *)malloc(gs->cap * sizeof(uint32_t));
        gs->old = (uint64_t *)malloc(gs->cap * width * sizeof(uint64_t));
        if (!gs->touched || !gs->old)
            return TNREF_ENOMEM;
    }
    /* snapshot the rows of the group's nodes */
    uint64_t nt = 0;
    for (uint64_t e = g0; e < g1; ++e) {
        uint32_t ends[2] = {u[e], v[e]};
        for (int q = 0; q < 2; ++q) {
            uint32_t x = ends[q];
            if (gs->slot[x] < 0) {
                gs->slot[x] = (int64_t)nt;
                gs->touched[nt] = x;
                memcpy(gs->old + nt * width, S + (uint64_t)x * width, width * sizeof(uint64_t));
                ++nt;
            }
        }
    }
    /* OR the partners' old rows into each endpoint */
    for (uint64_t e = g0; e < g1; ++e) {
        uint64_t *ra = S + (uint64_t)u[e] * width;
        uint64_t *rb = S + (uint64_t)v[e] * width;
        const uint64_t *oa = gs->old + (uint64_t)gs->slot[u[e]] * width;
        const uint64_t *ob = gs->old + (uint64_t)gs->slot[v[e]] * width;
        for (uint64_t w = 0; w < width; ++w) {
            ra[w] |= ob[w];
            rb[w] |= oa[w];
        }
    }
    for (uint64_t k = 0; k < nt; ++k)
        gs->slot[gs->touched[k]] = -1;
    return TNREF_OK;
}

/* Algorithm 1 with group snapshots, in chronological order (reverse = 0) or,
 * for the reversed-sequence variant of Section 3.4, from the last group to
 * the first (reverse = 1): then row i ends as the out-component of i. */
static int apply_events_dir(const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t m,
                            uint32_t n, uint64_t *S, uint64_t width, int reverse)
{
    if (m == 0)
        return TNREF_OK;
    int rc = tnref_validate(u, v, t, m, n);
    if (rc != TNREF_OK)
        return rc;
    struct tnref_groups gs = {NULL, NULL, NULL, 0};
    gs.slot = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!gs.slot)
        return TNREF_ENOMEM;
    for (uint32_t i = 0; i < n; ++i)
        gs.slot[i] = -1;
    if (!reverse) {
        uint64_t g0 = 0;
        while (g0 < m && rc == TNREF_OK) {
            uint64_t g1 = g0 + 1;
            while (g1 < m && t[g1] == t[g0])
                ++g1;
            rc = apply_group(&gs, u, v, g0, g1, S, width);
            g0 = g1;
        }
    } else {
        uint64_t g1 = m;
        while (g1 > 0 && rc == TNREF_OK) {
            uint64_t g0 = g1 - 1;
            while (g0 > 0 && t[g0 - 1] == t[g1 - 1])
                --g0;
            rc = apply_group(&gs, u, v, g0, g1, S, width);
            g1 = g0;
        }
    }
    free(gs.slot);
    free(gs.touched);
    free(gs.old);
    return rc;
}

/* Directed events (the paper's footnote to Section 3.1: only the receiving
 * node's row is updated, S[v] |= S[u]).  One timestamp group [g0, g1) is a
 * snapshot: S_new[v] = S_old[v] OR (OR over events u -> v of the group of
 * S_old[u]); the sources' old rows are copied first. */
static int apply_group_directed(struct tnref_groups *gs, const uint32_t *u, const uint32_t *v, uint64_t g0,
                                uint64_t g1, uint64_t *S, uint64_t width)
{
    uint64_t need = g1 - g0;
    if (need > gs->cap) {
        free(gs->touched);
        free(gs->old);
        gs->cap = need;
        gs->touched = (uint32_t *)malloc(gs->cap * sizeof(uint32_t));
        gs->old = (uint64_t *)malloc(gs->cap * width * sizeof(uint64_t));
        if (!gs->touched || !gs->old)
            return TNREF_ENOMEM;
    }
    uint64_t nt = 0;
    for (uint64_t e = g0; e < g1; ++e) {
        uint32_t x = u[e];
        if (gs->slot[x] < 0) {
            gs->slot[x] = (int64_t)nt;
            gs->touched[nt] = x;
            memcpy(gs->old + nt * width, S + (uint64_t)x * width, width * sizeof(uint64_t));
            ++nt;
        }
    }
    for (uint64_t e = g0; e < g1; ++e) {
        uint64_t *rv = S + (uint64_t)v[e] * width;
        const uint64_t *ou = gs->old + (uint64_t)gs->slot[u[e]] * width;
        for (uint64_t w = 0; w < width; ++w)
            rv[w] |= ou[w];
    }
    for (uint64_t k = 0; k < nt; ++k)
        gs->slot[gs->touched[k]] = -1;
    return TNREF_OK;
}

int tnref_apply_events_directed(const uint32_t *u, const uint32_t *v, const int64_t *t,
                                uint64_t m, uint32_t n, uint64_t *S, uint64_t width)
{
    if (m == 0)
        return TNREF_OK;
    int rc = tnref_validate(u, v, t, m, n);
    if (rc != TNREF_OK)
        return rc;
    struct tnref_groups gs = {NULL, NULL, NULL, 0};
    gs.slot = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!gs.slot)
        return TNREF_ENOMEM;
    for (uint32_t i = 0; i < n; ++i)
        gs.slot[i] = -1;
    uint64_t g0 = 0;
    while (g0 < m && rc == TNREF_OK) {
        uint64_t g1 = g0 + 1;
        while (g1 < m && t[g1] == t[g0])
            ++g1;
        rc = apply_group_directed(&gs, u, v, g0, g1, S, width);
        g0 = g1;
    }
    free(gs.slot);
    free(gs.touched);
    free(gs.old);
    return rc;
}

int tnref_apply_events(const uint32_t *u, const uint32_t *v, const int64_t *t,
                       uint64_t m, uint32_t n, uint64_t *S, uint64_t width)
{
    return apply_events_dir(u, v, t, m, n, S, width, 0);
}

int tnref_apply_events_reversed(const uint32_t *u, const uint32_t *v, const int64_t *t,
                                uint64_t m, uint32_t n, uint64_t *S, uint64_t width)
{
    return apply_events_dir(u, v, t, m, n, S, width, 1);
}

/* ---------------------------------------------------------------------------
 * Brute-force deterministic SI process from one source (Section 1: the
 * simple method that simulates spreading from every node at its first
 * appearance).  A susceptible node becomes infected when it interacts with a
 * node that was infected before the interaction's timestamp (equal timestamps
 * do not chain).  reached[i] = 1 iff node i is in the out-component of
 * `source`.  O(m) per source.
 * ------------------------------------------------------------------------- */
int tnref_si_reach(const uint32_t *u, const uint32_t *v, const int64_t *t,
                   uint64_t m, uint32_t n, uint32_t source, uint8_t *reached)
{
    if (source >= n)
        return TNREF_EINVAL;
    int rc = tnref_validate(u, v, t, m, n);
    if (rc != TNREF_OK)
        return rc;
    memset(reached, 0, n);
    reached[source] = 1;
    uint8_t *fresh = (uint8_t *)calloc(n, 1);
    if (!fresh)
        return TNREF_ENOMEM;
    uint64_t g0 = 0;
    while (g0 < m) {
        uint64_t g1 = g0 + 1;
        while (g1 < m && t[g1] == t[g0])
            ++g1;
        /* infections decided on the state before this timestamp */
        for (uint64_t e = g0; e < g1; ++e) {
            if (reached[u[e]])
                fresh[v[e]] = 1;
            if (reached[v[e]])
                fresh[u[e]] = 1;
        }
        for (uint64_t e = g0; e < g1; ++e) {
            if (fresh[u[e]]) {
                reached[u[e]] = 1;
                fresh[u[e]] = 0;
            }
            if (fresh[v[e]]) {
                reached[v[e]] = 1;
                fresh[v[e]] = 0;
            }
        }
        g0 = g1;
    }
    free(fresh);
    return TNREF_OK;
}

/* ---------------------------------------------------------------------------
 * Node growth (Section 3.5, advantages and limitations of the matrix method):
 * a node that joins the network brings a new row and a new column of zeros,
 * with only its own diagonal bit set.  S_old is n_old x n_old (row stride w_old
 * words), S_new is n_new x n_new (row stride w_new words), n_new >= n_old:
 *   S_new[i][j] = S_old[i][j]  for i, j < n_old,
 *   S_new[i][i] = 1            for n_old <= i < n_new,
 *   every other bit 0.
 * ------------------------------------------------------------------------- */
int tnref_grow_matrix(const uint64_t *S_old, uint32_t n_old, uint64_t w_old,
                      uint64_t *S_new, uint32_t n_new, uint64_t w_new)
{
    if (n_new < n_old || 64 * w_old < n_old || 64 * w_new < n_new) return TNREF_EINVAL;
    memset(S_new, 0, (size_t)n_new * w_new * sizeof(uint64_t));
    for (uint32_t i = 0; i < n_old; ++i)
        for (uint32_t j = 0; j < n_old; ++j)
            if ((S_old[(uint64_t)i * w_old + j / 64] >> (j % 64)) & 1u)
                S_new[(uint64_t)i * w_new + j / 64] |= 1ull << (j % 64);
    for (uint32_t i = n_old; i < n_new; ++i)
        S_new[(uint64_t)i * w_new + i / 64] |= 1ull << (i % 64);
    return TNREF_OK;
}

/* ---------------------------------------------------------------------------
 * Component sizes (Section 3, "count the number of ones in the corresponding
 * column"; eq. for s_t: row sums and column sums have the same total).
 * out[c] = number of rows with bit c set (out-component size of column c);
 * in[i]  = number of bits set in row i (in-component size of node i).
 * ------------------------------------------------------------------------- */
void tnref_column_counts(const uint64_t *S, uint32_t n_rows, uint64_t width,
                         uint64_t ncols, uint32_t *out)
{
    for (uint64_t c = 0; c < ncols; ++c) {
        uint32_t cnt = 0;
        for (uint32_t i = 0; i < n_rows; ++i)
            cnt += (uint32_t)((S[(uint64_t)i * width + c / 64] >> (c % 64)) & 1u);
        out[c] = cnt;
    }
}

void tnref_row_counts(const uint64_t *S, uint32_t n_rows, uint64_t width,
                      uint32_t *in)
{
    for (uint32_t i = 0; i < n_rows; ++i) {
        uint32_t cnt = 0;
        for (uint64_t c = 0; c < 64 * width; ++c)
            cnt += (uint32_t)((S[(uint64_t)i * width + c / 64] >> (c % 64)) & 1u);
        in[i] = cnt;
    }
}

/* Largest out-component: the first column index holding the maximum size. */
uint64_t tnref_argmax(const uint32_t *sizes, uint64_t count)
{
    uint64_t best = 0;
    for (uint64_t c = 1; c < count; ++c)
        if (sizes[c] > sizes[best])
            best = c;
    return best;
}

/* ---------------------------------------------------------------------------
 * Network hashing (Section 4.1).
 *
 * Prime p = 2^61 - 1, order 4 (degree-3 polynomials: 4-universal tables).
 * Coefficients A(i, c), i in {0,1,2}, c in [0, 4):
 *     A(i, c) = ((r1 << 32) + r2) mod p,   r = rand(2^31 - 1).
 * rand is read as a SplitMix64 stream reduced modulo 2^31 - 1.  Replica j's
 * stream starts from state splitmix64(seed XOR j); draws are taken in the
 * order i = 0..2, c = 0..3, r1 before r2.
 * Table value T_i[x]: start from A(i, 0) and apply acc <- (x * acc + A(i, c))
 * mod p for c = 1..3 (the MultAddMod recursion, order - 1 = 3 times).
 * Key split for a 32-bit node id u: x0 = u & 0xFFFF, x1 = u >> 16,
 * x2 = x0 + x1 (a 17-bit derived character, no wrap).
 * h(u) = (T0[x0] XOR T1[x1] XOR T2[x2]) mod k.
 * ------------------------------------------------------------------------- */
#define TNREF_P61 ((1ull << 61) - 1)

static uint64_t splitmix64_next(uint64_t *state)
{
    /* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
     * number generators", OOPSLA 2014): Weyl increment then a finaliser. */
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* The first `count` outputs of the generator started at `state` (exported so
 * that the tests can check it against the generator's known-answer values). */
void tnref_splitmix64_stream(uint64_t state, uint64_t count, uint64_t *out)
{
    for (uint64_t i = 0; i < count; ++i)
        out[i] = splitmix64_next(&state);
}

void tnref_hash_coeffs(uint64_t seed, uint32_t replica, uint64_t A[12])
{
    uint64_t st = seed ^ (uint64_t)replica;
    uint64_t stream = splitmix64_next(&st);
    for (int i = 0; i < 3; ++i) {
        for (int c = 0; c < 4; ++c) {
            uint64_t r1 = splitmix64_next(&stream) % 2147483647ull;
            uint64_t r2 = splitmix64_next(&stream) % 2147483647ull;
            A[i * 4 + c] = ((r1 << 32) + r2) % TNREF_P61;
        }
    }
}

uint64_t tnref_table_value(const uint64_t *Ai, uint64_t x)
{
    unsigned __int128 acc = Ai[0];
    for (int c = 1; c < 4; ++c)
        acc = (acc * x + Ai[c]) % TNREF_P61;
    return (uint64_t)acc;
}

uint64_t tnref_hash_raw(const uint64_t A[12], uint32_t u)
{
    uint64_t x0 = u & 0xFFFFu, x1 = u >> 16, x2 = x0 + x1;
    return tnref_table_value(A + 0, x0) ^ tnref_table_value(A + 4, x1) ^
           tnref_table_value(A + 8, x2);
}

/* H[j*n + x] = h_j(x) for replicas j < R and nodes x < n. */
int tnref_hash_nodes(uint64_t seed, uint32_t R, uint32_t k, uint32_t n,
                     uint32_t *H)
{
    if (k == 0)
        return TNREF_EINVAL;
    for (uint32_t j = 0; j < R; ++j) {
        uint64_t A[12];
        tnref_hash_coeffs(seed, j, A);
        for (uint32_t x = 0; x < n; ++x)
            H[(uint64_t)j * n + x] = (uint32_t)(tnref_hash_raw(A, x) % k);
    }
    return TNREF_OK;
}

/* Super-events (h(u), h(v), t) of one hashed network (Section 4.1). */
void tnref_proxy_events(const uint32_t *u, const uint32_t *v, uint64_t m,
                        const uint32_t *Hj, uint32_t *pu, uint32_t *pv)
{
    for (uint64_t e = 0; e < m; ++e) {
        pu[e] = Hj[u[e]];
        pv[e] = Hj[v[e]];
    }
}

/* ---------------------------------------------------------------------------
 * Fusion (Section 4.2, eqs. DefInvHComp and DefEstOCMerge):
 *   est(u) = | intersection over j of h_j^{-1}( OC_j( h_j(u) ) ) |.
 * Node w lies in h_j^{-1}(OC_j(b)) exactly when super-node h_j(w) is reached
 * from super-node b in proxy j, i.e. bit b of row h_j(w) of P_j is set.
 * P holds R proxy matrices, each k rows of wk = ceil(k/64) words.  Sources are
 * src[0..nsrc) (or all n nodes when src == NULL).  O(n * nsrc * R).
 * ------------------------------------------------------------------------- */
int tnref_hash_estimate(const uint64_t *P, uint32_t R, uint32_t k,
                        const uint32_t *H, uint32_t n, const uint32_t *src,
                        uint64_t nsrc, uint32_t *est)
{
    uint64_t wk = (k + 63) / 64;
    uint64_t count = src ? nsrc : n;
    for (uint64_t s = 0; s < count; ++s) {
        uint32_t x = src ? src[s] : (uint32_t)s;
        if (x >= n)
            return TNREF_ERANGE;
        uint32_t c = 0;
        for (uint32_t w = 0; w < n; ++w) {
            int in_all = 1;
            for (uint32_t j = 0; j < R && in_all; ++j) {
                uint32_t b = H[(uint64_t)j * n + x];
                uint32_t row = H[(uint64_t)j * n + w];
                const uint64_t *Pj = P + (uint64_t)j * k * wk;
                in_all = (int)((Pj[(uint64_t)row * wk + b / 64] >> (b % 64)) & 1u);
            }
            c += (uint32_t)in_all;
        }
        est[s] = c;
    }
    return TNREF_OK;
}

/* ---------------------------------------------------------------------------
 * Error of the hashed estimate against the exact sizes (Section 4.4 compares
 * the estimated and the exact out-component size distributions with the
 * Earth-Mover distance).  For two samples a (estimates) and b (exact sizes) of
 * the same sources, count entries each:
 *   sum_abs = sum |a_s - b_s|,        max_abs = max |a_s - b_s|,
 *   rel_sum = sum |a_s - b_s| / b_s,  max_rel = max |a_s - b_s| / b_s
 *   (in double, summed in source order; b_s >= 1 since a node reaches itself),
 *   w1_num  = sum_i |sort(a)_i - sort(b)_i|, i.e. count * W1 between the two
 *   empirical distributions (for equal-size samples the optimal transport
 *   plan matches the sorted orders).
 * Returns TNREF_EINVAL if an exact size is 0.
 * ------------------------------------------------------------------------- */
static int cmp_u32(const void *x, const void *y)
{
    uint32_t a = *(const uint32_t *)x, b = *(const uint32_t *)y;
    return (a > b) - (a < b);
}

int tnref_error_stats(const uint32_t *a, const uint32_t *b, uint64_t count,
                      uint64_t *sum_abs, uint64_t *max_abs, uint64_t *w1_num,
                      double *rel_sum, double *max_rel)
{
    uint64_t s = 0, mx = 0, w = 0;
    double rs = 0.0, mr = 0.0;
    for (uint64_t i = 0; i < count; ++i) {
        if (b[i] == 0)
            return TNREF_EINVAL;
        uint64_t d = a[i] > b[i] ? (uint64_t)(a[i] - b[i]) : (uint64_t)(b[i] - a[i]);
        s += d;
        if (d > mx)
            mx = d;
        double r = (double)d / (double)b[i];
        rs += r;
        if (r > mr)
            mr = r;
    }
    uint32_t *sa = malloc(count * sizeof(uint32_t) + 1);
    uint32_t *sb = malloc(count * sizeof(uint32_t) + 1);
    if (!sa || !sb) {
        free(sa);
        free(sb);
        return TNREF_ENOMEM;
    }
    memcpy(sa, a, count * sizeof(uint32_t));
    memcpy(sb, b, count * sizeof(uint32_t));
    qsort(sa, count, sizeof(uint32_t), cmp_u32);
    qsort(sb, count, sizeof(uint32_t), cmp_u32);
    for (uint64_t i = 0; i < count; ++i)
        w += sa[i] > sb[i] ? (uint64_t)(sa[i] - sb[i]) : (uint64_t)(sb[i] - sa[i]);
    free(sa);
    free(sb);
    *sum_abs = s;
    *max_abs = mx;
    *w1_num = w;
    *rel_sum = rs;
    *max_rel = mr;
    return TNREF_OK;
}

/* Deterministic SI over directed events: an infected u infects v at the
 * event's time (infections of one timestamp are decided on the state before
 * it). */
int tnref_si_reach_directed(const uint32_t *u, const uint32_t *v, const int64_t *t,
                            uint64_t m, uint32_t n, uint32_t source, uint8_t *reached)
{
    if (source >= n)
        return TNREF_EINVAL;
    int rc = tnref_validate(u, v, t, m, n);
    if (rc != TNREF_OK)
        return rc;
    memset(reached, 0, n);
    reached[source] = 1;
    uint8_t *fresh = (uint8_t *)calloc(n, 1);
    if (!fresh)
        return TNREF_ENOMEM;
    uint64_t g0 = 0;
    while (g0 < m) {
        uint64_t g1 = g0 + 1;
        while (g1 < m && t[g1] == t[g0])
            ++g1;
        for (uint64_t e = g0; e < g1; ++e)
            if (reached[u[e]])
                fresh[v[e]] = 1;
        for (uint64_t e = g0; e < g1; ++e)
            if (fresh[v[e]]) {
                reached[v[e]] = 1;
                fresh[v[e]] = 0;
            }
        g0 = g1;
    }
    free(fresh);
    return TNREF_OK;
}

/* ---------------------------------------------------------------------------
 * HyperLogLog sketches of the components (Section 3.3, and Section 3.4 with
 * the reversed sequence; Flajolet, Fusy,
 * Gandouet, Meunier 2007).  Each node keeps s = 2^p one-byte registers.  An
 * element x hashes to h = one SplitMix64 step from state (seed XOR x); its
 * register is the top p bits of h and its rank the position of the first 1 in
 * the remaining 64 - p bits (64 - p + 1 if they are all 0).  Node i starts as
 * the sketch of {i}; an event merges sketches by register-wise maximum with
 * the same snapshot rule per timestamp group as the component matrix, so that
 * node i's sketch is always the sketch of its in-component (of its
 * out-component when the sequence is processed in reverse).  The estimate of
 * a sketch M is E = alpha_s s^2 / sum_j 2^(-M[j]), replaced by linear counting
 * s ln(s / V) when E <= 2.5 s and V > 0 registers are zero.
 * ------------------------------------------------------------------------- */
void tnref_hll_singleton(uint64_t seed, uint32_t p, uint32_t x, uint32_t *reg, uint8_t *rank)
{
    uint64_t st = seed ^ (uint64_t)x;
    uint64_t h = splitmix64_next(&st);
    *reg = (uint32_t)(h >> (64 - p));
    uint64_t w = h << p;
    uint32_t r = 1;
    while (r <= 64 - p && !(w & (1ull << 63))) {
        ++r;
        w <<= 1;
    }
    *rank = (uint8_t)r;
}

static void hll_merge_group(const uint32_t *u, const uint32_t *v, uint64_t g0, uint64_t g1, uint8_t *R,
                            uint32_t s, int directed, int turn, uint8_t *old, int64_t *slot,
                            uint32_t *touched)
{
    uint64_t nt = 0;
    for (uint64_t e = g0; e < g1; ++e) {
        uint32_t a = turn ? v[e] : u[e], b = turn ? u[e] : v[e];
        uint32_t ends[2] = {a, b};
        for (int q = 0; q < (directed ? 1 : 2); ++q) { /* rows that are read: senders (directed) or both ends */
            uint32_t x = ends[q];
            if (slot[x] < 0) {
                slot[x] = (int64_t)nt;
                touched[nt] = x;
                memcpy(old + nt * s, R + (uint64_t)x * s, s);
                ++nt;
            }
        }
    }
    for (uint64_t e = g0; e < g1; ++e) {
        uint32_t a = turn ? v[e] : u[e], b = turn ? u[e] : v[e];
        uint8_t *rb = R + (uint64_t)b * s;
        const uint8_t *oa = old + (uint64_t)slot[a] * s;
        for (uint32_t j = 0; j < s; ++j)
            if (oa[j] > rb[j])
                rb[j] = oa[j];
        if (!directed) {
            uint8_t *ra = R + (uint64_t)a * s;
            const uint8_t *ob = old + (uint64_t)slot[b] * s;
            for (uint32_t j = 0; j < s; ++j)
                if (ob[j] > ra[j])
                    ra[j] = ob[j];
        }
    }
    for (uint64_t k = 0; k < nt; ++k)
        slot[touched[k]] = -1;
}

/* R: n x 2^p registers.  reverse: groups from the last to the first (and
 * directed events turned around), so row i sketches the out-component of i. */
int tnref_hll_sketches(const uint32_t *u, const uint32_t *v, const int64_t *t, uint64_t m, uint32_t n,
                       uint32_t p, uint64_t seed, int reverse, int directed, uint8_t *R)
{
    if (p < 4 || p > 16)
        return TNREF_EINVAL;
    int rc = tnref_validate(u, v, t, m, n);
    if (rc != TNREF_OK)
        return rc;
    const uint32_t s = 1u << p;
    memset(R, 0, (size_t)n * s);
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t reg;
        uint8_t rank;
        tnref_hll_singleton(seed, p, i, &reg, &rank);
        R[(uint64_t)i * s + reg] = rank;
    }
    if (m == 0)
        return TNREF_OK;
    int64_t *slot = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    uint32_t *touched = (uint32_t *)malloc(2 * m * sizeof(uint32_t));
    uint8_t *old = (uint8_t *)malloc(2 * m * (size_t)s);
    if (!slot || !touched || !old) {
        free(slot);
        free(touched);
        free(old);
        return TNREF_ENOMEM;
    }
    for (uint32_t i = 0; i < n; ++i)
        slot[i] = -1;
    const int turn = reverse && directed;
    if (!reverse) {
        uint64_t g0 = 0;
        while (g0 < m) {
            uint64_t g1 = g0 + 1;
            while (g1 < m && t[g1] == t[g0])
                ++g1;
            hll_merge_group(u, v, g0, g1, R, s, directed, turn, old, slot, touched);
            g0 = g1;
        }
    } else {
        uint64_t g1 = m;
        while (g1 > 0) {
            uint64_t g0 = g1 - 1;
            while (g0 > 0 && t[g0 - 1] == t[g1 - 1])
                --g0;
            hll_merge_group(u, v, g0, g1, R, s, directed, turn, old, slot, touched);
            g1 = g0;
        }
    }
    free(slot);
    free(touched);
    free(old);
    return TNREF_OK;
}

void tnref_hll_estimate(const uint8_t *R, uint32_t n, uint32_t p, double *est)
{
    const uint32_t s = 1u << p;
    double alpha;
    if (s == 16)
        alpha = 0.673;
    else if (s == 32)
        alpha = 0.697;
    else if (s == 64)
        alpha = 0.709;
    else
        alpha = 0.7213 / (1.0 + 1.079 / (double)s);
    for (uint32_t i = 0; i < n; ++i) {
        const uint8_t *M = R + (uint64_t)i * s;
        double z = 0.0;
        uint32_t zeros = 0;
        for (uint32_t j = 0; j < s; ++j) {
            z += ldexp(1.0, -(int)M[j]);
            zeros += M[j] == 0;
        }
        double e = alpha * (double)s * (double)s / z;
        if (e <= 2.5 * (double)s && zeros > 0)
            e = (double)s * log((double)s / (double)zeros);
        est[i] = e;
    }
}
