/*
 * rmq_oracle.c -- CPU oracle for batched range minimum queries (RMQ).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the GPU library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark load it.  The
 * GPU library never calls, links or includes anything from here, and this
 * file includes nothing from the GPU library.
 *
 * Source: S. Grabowski, T. Kowalski, "Faster batched range minimum queries"
 * (arXiv:1706.06940).  Conventions taken for this library:
 *   - 0-based positions, inclusive ranges [l, r]      (paper: 1-based, Sec. 1)
 *   - ties resolved to the LEFTMOST minimum position  (paper: Sec. 1 mentions
 *     this variant; the library fixes it so that results are unique)
 *   - a query with l < 0, r >= n or l > r is invalid and answers -1
 *     (the library's per-query error contract; the paper's generator swaps
 *     l and r, the API does not).
 *
 * Every function works on positions (int32) and values (int32); none of the
 * GPU path's encodings (packed keys, block tables in memory) appears here.
 *
 * Pins (tests/test_oracle_pins.py): exhaustive brute force on tiny arrays,
 * invariants, closed forms, numpy library routines (argmin, lexsort,
 * searchsorted) on the step-level functions, and planted mutants that the
 * pins must reject.  No function here is "parity unpinned".
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_API __attribute__((visibility("default")))

static int valid_query(int64_t n, int32_t l, int32_t r)
{
    return l >= 0 && r >= l && (int64_t)r < n;
}

/* Number of OpenMP threads the oracle will use (1 without OpenMP). */
ORACLE_API int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * The RMQ definition (Sec. 1): RMQ_A(i, j) = argmin_{i<=t<=j} A[t], answered
 * by the trivial per-query scan the paper names as the online cost
 * O(r_i - l_i + 1) (Sec. 1).  The scan keeps the first strictly smaller
 * value, which yields the leftmost minimum.  Parallel over queries only.
 */
ORACLE_API void oracle_rmq_naive(const int32_t *A, int64_t n,
                                 const int32_t *l, const int32_t *r, int64_t q,
                                 int32_t *out, int nthreads)
{
    int64_t i;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (i = 0; i < q; ++i) {
        int32_t lo = l[i], hi = r[i];
        if (!valid_query(n, lo, hi)) { out[i] = -1; continue; }
        int32_t best = lo;
        for (int64_t t = (int64_t)lo + 1; t <= hi; ++t)
            if (A[t] < A[best]) best = (int32_t)t;
        out[i] = best;
    }
    (void)nthreads;
}

/* floor(log2(x)) for x >= 1 */
static int ilog2_u64(uint64_t x)
{
    int t = -1;
    while (x) { x >>= 1; ++t; }
    return t;
}

/* Leftmost-minimum choice between two candidate positions a <= b. */
static int32_t pick_left(const int32_t *A, int32_t a, int32_t b)
{
    return (A[a] <= A[b]) ? a : b;
}

/* Number of levels of a textbook sparse table over m items: floor(log2 m)+1. */
ORACLE_API int oracle_sparse_levels(int64_t m)
{
    return m <= 0 ? 0 : ilog2_u64((uint64_t)m) + 1;
}

/*
 * Textbook Sparse Table (Bender and Farach, recalled in Sec. 2): for every
 * left end i and every t, M[t][i] is the position of the minimum of
 * A[i .. i + 2^t - 1]; a query [i, j] is the smaller of the two overlapping
 * windows A[i .. i+2^t'-1] and A[j-2^t'+1 .. j] with t' = floor(log(j - i))
 * (Sec. 2).  i == j is answered directly.  Combines prefer the left
 * candidate on equal values, which keeps the leftmost minimum.
 *
 * Exact like the naive scan, it serves as the scalable checker: its cost is
 * O(n log n) build + O(1) per query instead of O(r - l + 1) per query.
 * Memory: (floor(log2 n)+1) * 4n bytes, allocated here and freed on return.
 * Returns 0 on success, -1 if the table cannot be allocated.
 */
ORACLE_API int oracle_rmq_sparse_table(const int32_t *A, int64_t n,
                                       const int32_t *l, const int32_t *r, int64_t q,
                                       int32_t *out, int nthreads)
{
    if (n <= 0) {
        for (int64_t i = 0; i < q; ++i) out[i] = -1;
        return 0;
    }
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#endif
    int levels = oracle_sparse_levels(n);
    int32_t **M = (int32_t **)calloc((size_t)levels, sizeof(int32_t *));
    if (!M) return -1;
    for (int t = 0; t < levels; ++t) {
        M[t] = (int32_t *)malloc((size_t)n * sizeof(int32_t));
        if (!M[t]) {
            for (int u = 0; u < t; ++u) free(M[u]);
            free(M);
            return -1;
        }
    }
    int64_t i;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
    for (i = 0; i < n; ++i) M[0][i] = (int32_t)i;
    for (int t = 1; t < levels; ++t) {
        int64_t half = (int64_t)1 << (t - 1);
        int64_t cnt = n - ((int64_t)1 << t) + 1;
        int32_t *prev = M[t - 1], *cur = M[t];
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
        for (i = 0; i < cnt; ++i) cur[i] = pick_left(A, prev[i], prev[i + half]);
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
    for (i = 0; i < q; ++i) {
        int32_t lo = l[i], hi = r[i];
        if (!valid_query(n, lo, hi)) { out[i] = -1; continue; }
        if (lo == hi) { out[i] = lo; continue; }
        int t = ilog2_u64((uint64_t)(hi - lo));          /* t' = floor(log(j - i)) */
        int32_t a = M[t][lo];
        int32_t b = M[t][(int64_t)hi - ((int64_t)1 << t) + 1];
        out[i] = pick_left(A, a, b);
    }
    for (int t = 0; t < levels; ++t) free(M[t]);
    free(M);
    (void)nthreads;
    return 0;
}

/* Leftmost minimum position of A[lo .. hi] (inclusive), by plain scan. */
static int32_t scan_min(const int32_t *A, int64_t lo, int64_t hi)
{
    int64_t best = lo;
    for (int64_t t = lo + 1; t <= hi; ++t)
        if (A[t] < A[best]) best = t;
    return (int32_t)best;
}

/*
 * Step 3 of BbST, level 0 (Sec. 3.1 step 3 and Sec. 3.2): split A into blocks
 * of k cells, block j = A[j*k .. min(n, (j+1)*k) - 1] (the last block may be
 * short), and report the position of each block's minimum.
 * pos_out has ceil(n / k) entries.
 */
ORACLE_API void oracle_block_minima(const int32_t *A, int64_t n, int64_t k, int32_t *pos_out)
{
    int64_t nb = (n + k - 1) / k;
    for (int64_t j = 0; j < nb; ++j) {
        int64_t lo = j * k, hi = lo + k - 1;
        if (hi > n - 1) hi = n - 1;
        pos_out[j] = scan_min(A, lo, hi);
    }
}

/*
 * Step 3 of BbST, all levels (Sec. 3.1 step 3): for each block B_j and each
 * level t = 0 .. floor(log2 nb), the position of the minimum over the span of
 * 2^t consecutive blocks whose leftmost block is B_j, i.e. over
 * A[j*k .. min(n, (j + 2^t)*k) - 1].  Only spans that end inside the block
 * range (j + 2^t <= nb) exist; other slots are set to -1.
 *
 * Written as the definition (a direct scan of each span), not by doubling,
 * so that it checks the GPU path's doubling independently.
 * T has levels * nb entries, level-major: T[t * nb + j].
 */
ORACLE_API void oracle_block_sparse_table(const int32_t *A, int64_t n, int64_t k, int32_t *T)
{
    int64_t nb = (n + k - 1) / k;
    int levels = oracle_sparse_levels(nb);
    for (int t = 0; t < levels; ++t) {
        int64_t span = (int64_t)1 << t;
        for (int64_t j = 0; j < nb; ++j) {
            if (j + span > nb) { T[(int64_t)t * nb + j] = -1; continue; }
            int64_t lo = j * k, hi = (j + span) * k - 1;
            if (hi > n - 1) hi = n - 1;
            T[(int64_t)t * nb + j] = scan_min(A, lo, hi);
        }
    }
}

typedef struct { uint32_t pos; uint32_t tag; } endpoint_t;

static int cmp_endpoint(const void *x, const void *y)
{
    const endpoint_t *a = (const endpoint_t *)x, *b = (const endpoint_t *)y;
    if (a->pos != b->pos) return a->pos < b->pos ? -1 : 1;
    if (a->tag != b->tag) return a->tag < b->tag ? -1 : 1;
    return 0;
}

/*
 * Step 1 of BbST_CON (Sec. 3.1 step 1): each of the 2q endpoints is a pair
 * (position in A, index in the query list); sorting by position yields the
 * list E[1 .. 2q] with non-decreasing positions.  The satellite is encoded
 * as tag = 2*i + side (side 0 = l_i, 1 = r_i).  Equal positions keep the
 * input order (ascending tag), i.e. this is the stable sort of the sequence
 * l_0, r_0, l_1, r_1, ...  Invalid queries are not filtered here.
 * pos_out / tag_out have 2q entries.  Returns 0, or -1 on allocation failure.
 */
ORACLE_API int oracle_sort_endpoints(const int32_t *l, const int32_t *r, int64_t q,
                                     uint32_t *pos_out, uint32_t *tag_out)
{
    endpoint_t *e = (endpoint_t *)malloc((size_t)(2 * q > 0 ? 2 * q : 1) * sizeof(endpoint_t));
    if (!e) return -1;
    for (int64_t i = 0; i < q; ++i) {
        e[2 * i].pos = (uint32_t)l[i];
        e[2 * i].tag = (uint32_t)(2 * i);
        e[2 * i + 1].pos = (uint32_t)r[i];
        e[2 * i + 1].tag = (uint32_t)(2 * i + 1);
    }
    qsort(e, (size_t)(2 * q), sizeof(endpoint_t), cmp_endpoint);
    for (int64_t i = 0; i < 2 * q; ++i) { pos_out[i] = e[i].pos; tag_out[i] = e[i].tag; }
    free(e);
    return 0;
}

/*
 * Remapping of step 1 (Sec. 3.1 step 1, "remap them with respect to the
 * contracted array's indices"): from the sorted endpoint list, P[0 .. m) are
 * the distinct endpoint positions in increasing order, and every query gets
 * the indices a_i, b_i with P[a_i] = l_i and P[b_i] = r_i.  Duplicate
 * positions collapse to one entry (the paper calls their effect negligible,
 * Sec. 2; collapsing them does not change any answer).
 * Returns m.
 */
ORACLE_API int64_t oracle_rank_endpoints(const uint32_t *pos_sorted, const uint32_t *tag_sorted,
                                         int64_t cnt, uint32_t *P_out,
                                         int32_t *rank_l, int32_t *rank_r)
{
    int64_t m = 0;
    for (int64_t i = 0; i < cnt; ++i) {
        if (i == 0 || pos_sorted[i] != pos_sorted[i - 1]) P_out[m++] = pos_sorted[i];
        int32_t rank = (int32_t)(m - 1);
        uint32_t tag = tag_sorted[i];
        if (tag & 1u) rank_r[tag >> 1] = rank;
        else rank_l[tag >> 1] = rank;
    }
    return m;
}

/*
 * Step 2 of BbST_CON (Sec. 3.1 step 2): A_Q[j] is the minimum of the area
 * A[P_j .. P_{j+1}] (both ends included, so consecutive areas share their
 * endpoint), j = 0 .. m-2.  Reported as the position of the leftmost
 * minimum, which also plays the role of the paper's helper array mapping
 * A_Q indices back to positions in A.  pos_out has m-1 entries.
 */
ORACLE_API void oracle_contract(const int32_t *A, int64_t n, const uint32_t *P, int64_t m,
                                int32_t *pos_out)
{
    (void)n;
    for (int64_t j = 0; j + 1 < m; ++j) pos_out[j] = scan_min(A, (int64_t)P[j], (int64_t)P[j + 1]);
}

/*
 * Step 4 applied to the contracted array (Sec. 3.1 step 4), written as the
 * definition over A_Q: with a = rank of l, b = rank of r, the query covers
 * the areas j = a .. b-1, whose union is [l, r]; its answer is the leftmost
 * minimum over those area minima (compared by value, then by position).
 * When a == b (l == r) the answer is l.  AQ_pos holds positions in A
 * (from oracle_contract); invalid queries answer -1.
 */
ORACLE_API void oracle_contracted_query(const int32_t *A, int64_t n,
                                        const int32_t *AQ_pos,
                                        const int32_t *l, const int32_t *r,
                                        const int32_t *rank_l, const int32_t *rank_r,
                                        int64_t q, int32_t *out)
{
    for (int64_t i = 0; i < q; ++i) {
        if (!valid_query(n, l[i], r[i])) { out[i] = -1; continue; }
        int32_t a = rank_l[i], b = rank_r[i];
        if (a == b) { out[i] = l[i]; continue; }
        int32_t best = AQ_pos[a];
        for (int32_t j = a + 1; j < b; ++j) {
            int32_t p = AQ_pos[j];
            if (A[p] < A[best] || (A[p] == A[best] && p < best)) best = p;
        }
        out[i] = best;
    }
}

/* The candidate with the smaller value, and of equal values the one more to
 * the left (candidates in any order). */
static int32_t lex_min(const int32_t *A, int32_t a, int32_t b)
{
    if (A[a] != A[b]) return A[a] < A[b] ? a : b;
    return a < b ? a : b;
}

/*
 * The l-ary generalisation of the block sparse table (Sec. 3.1, the variant
 * the paper describes but does not implement): level t holds, for each
 * block B_j, the minimum over the l^t consecutive blocks whose leftmost
 * block is B_j; levels t = 0 .. floor(log_l nb).  For l = 2 this is the
 * block sparse table above.
 */
ORACLE_API int oracle_lary_levels(int64_t nb, int64_t ell)
{
    if (nb <= 0 || ell < 2) return 0;
    int levels = 1;
    for (int64_t span = ell; span <= nb; span *= ell) ++levels;
    return levels;
}

/*
 * The l-ary table written as its definition (a direct scan of each span).
 * T has levels * nb entries, level-major; spans that would end past the
 * last block are -1.
 */
ORACLE_API void oracle_lary_block_table(const int32_t *A, int64_t n, int64_t k, int64_t ell, int32_t *T)
{
    int64_t nb = (n + k - 1) / k;
    int levels = oracle_lary_levels(nb, ell);
    int64_t span = 1;
    for (int t = 0; t < levels; ++t, span *= ell) {
        for (int64_t j = 0; j < nb; ++j) {
            if (j + span > nb) { T[(int64_t)t * nb + j] = -1; continue; }
            int64_t lo = j * k, hi = (j + span) * k - 1;
            if (hi > n - 1) hi = n - 1;
            T[(int64_t)t * nb + j] = scan_min(A, lo, hi);
        }
    }
}

/*
 * Queries over the l-ary table, in the steps of Sec. 3.1 step 4 with the
 * variant's lookup: blocks bl = l / k and br = r / k; a query inside one
 * block is scanned.  Otherwise the inner span of blocks bl+1 .. br-1, of
 * length len, is covered by spans of the level t = floor(log_l len), of
 * l^t blocks each, placed from bl+1 and then one more ending at br-1, so
 * that at most l table values are compared.  The two end parts are scanned,
 * and the leftmost minimum of the three parts is the answer.  T comes from
 * oracle_lary_block_table; lookups[i] (may be NULL) receives the number of
 * table values used.  Invalid queries answer -1.
 */
ORACLE_API void oracle_lary_query(const int32_t *A, int64_t n, int64_t k, int64_t ell, const int32_t *T,
                                  const int32_t *l, const int32_t *r, int64_t q, int32_t *out,
                                  int32_t *lookups)
{
    int64_t nb = (n + k - 1) / k;
    for (int64_t i = 0; i < q; ++i) {
        int32_t used = 0;
        if (!valid_query(n, l[i], r[i])) {
            out[i] = -1;
            if (lookups) lookups[i] = 0;
            continue;
        }
        int64_t bl = l[i] / k, br = r[i] / k;
        if (bl == br) {
            out[i] = scan_min(A, l[i], r[i]);
            if (lookups) lookups[i] = 0;
            continue;
        }
        int32_t best = scan_min(A, l[i], (bl + 1) * k - 1);   /* left end part */
        if (br - bl >= 2) {
            int64_t a = bl + 1, b = br - 1, len = b - a + 1;
            int t = 0;
            int64_t span = 1;
            while (span * ell <= len) { span *= ell; ++t; }
            for (int64_t s = a;; s += span) {
                int64_t start = s + span - 1 <= b ? s : b - span + 1;   /* the last one ends at b */
                best = lex_min(A, best, T[(int64_t)t * nb + start]);
                ++used;
                if (start + span - 1 >= b) break;
            }
        }
        best = lex_min(A, best, scan_min(A, br * k, r[i]));   /* right end part */
        out[i] = best;
        if (lookups) lookups[i] = used;
    }
}

/*
 * The multi-level block-based sparse table of Sec. 3.3: block sizes
 * k_1 < k_2 < ... < k_h, each dividing the next.  The minima of the
 * non-overlapping blocks of size k_i are kept for 1 <= i < h, and for
 * blocks of size k_h their minima, doubles, quadruples and so on (the
 * sparse table of Sec. 3.1 step 3 over blocks of k_h).  Space in entries:
 * n/k_1 + ... + n/k_{h-1} + (n/k_h)(floor(log2(n/k_h)) + 1), block counts
 * rounded up.  ks[0 .. h-1] = k_1 .. k_h.  Returns -1 on bad parameters
 * (h < 1, k_1 < 1, or some k_i not dividing k_{i+1}).
 */
ORACLE_API int64_t oracle_hlevel_space(int64_t n, const int64_t *ks, int h)
{
    if (n <= 0 || h < 1 || ks[0] < 1) return -1;
    for (int i = 0; i + 1 < h; ++i)
        if (ks[i + 1] <= ks[i] || ks[i + 1] % ks[i] != 0) return -1;
    int64_t words = 0;
    for (int i = 0; i + 1 < h; ++i) words += (n + ks[i] - 1) / ks[i];
    int64_t nb = (n + ks[h - 1] - 1) / ks[h - 1];
    return words + nb * oracle_sparse_levels(nb);
}

/*
 * Leftmost minimum position of A[a .. b], a part lying inside one block of
 * level lev (blocks of ks[lev - 1] cells; M[i - 1] holds the minima of the
 * blocks of level i, i < h).  At level 1 the part is scanned.  Otherwise the
 * blocks of level lev - 1 lying wholly inside the part give their minima, and
 * the cells before the first and after the last of them form at most two
 * parts of level lev - 1, resolved one level down: the "checking of up to
 * two blocks" of Sec. 3.3, at cost k_lev / k_{lev-1} per level and k_1 at the
 * bottom.  *work counts the cells scanned and the minima read.
 */
static int32_t hlevel_part(const int32_t *A, int32_t *const *M, const int64_t *ks, int lev, int64_t a, int64_t b,
                           int64_t *work)
{
    if (lev == 1) {
        *work += b - a + 1;
        return scan_min(A, a, b);
    }
    int64_t s = ks[lev - 2];           /* block size of level lev - 1 */
    int64_t first = (a + s - 1) / s;   /* first block of level lev - 1 starting at or after a */
    int64_t last = (b + 1) / s;        /* blocks first .. last - 1 end at or before b */
    if (first >= last) {               /* no whole block inside: one or two parts one level down */
        if (a / s == b / s) return hlevel_part(A, M, ks, lev - 1, a, b, work);
        int32_t x = hlevel_part(A, M, ks, lev - 1, a, (a / s + 1) * s - 1, work);
        return lex_min(A, x, hlevel_part(A, M, ks, lev - 1, (b / s) * s, b, work));
    }
    int32_t best = -1;
    if (a < first * s) best = hlevel_part(A, M, ks, lev - 1, a, first * s - 1, work);
    for (int64_t j = first; j < last; ++j) {
        int32_t p = M[lev - 2][j];
        best = best < 0 ? p : lex_min(A, best, p);
        ++*work;
    }
    if (last * s <= b) best = lex_min(A, best, hlevel_part(A, M, ks, lev - 1, last * s, b, work));
    return best;
}

/*
 * Queries over the multi-level structure (Sec. 3.3), in the paper's order:
 * the block minima of every level i < h, written as their definition (a scan
 * of each block); the sparse table over blocks of k_h (a scan of each span);
 * then each query: with bl = l / k_h and br = r / k_h, the inner span of
 * blocks bl+1 .. br-1 from two overlapping table lookups at level
 * t = floor(log2(br - bl - 1)) (Sec. 3.1 step 4), and the two end parts, each
 * inside one block of k_h, resolved down the levels (hlevel_part); a query
 * inside one block of k_h is one such part.  work (may be NULL) receives per
 * query the cells scanned, minima read and table values used.  Returns -1 on
 * bad parameters or when memory cannot be had.  Invalid queries answer -1.
 */
ORACLE_API int oracle_hlevel_query(const int32_t *A, int64_t n, const int64_t *ks, int h,
                                   const int32_t *l, const int32_t *r, int64_t q, int32_t *out, int64_t *work)
{
    if (oracle_hlevel_space(n, ks, h) < 0 || h > 16) return -1;
    int32_t *M[16] = {0};
    int rc = 0;
    for (int i = 0; i + 1 < h && rc == 0; ++i) {
        int64_t nbi = (n + ks[i] - 1) / ks[i];
        M[i] = (int32_t *)malloc((size_t)nbi * sizeof(int32_t));
        if (!M[i]) { rc = -1; break; }
        oracle_block_minima(A, n, ks[i], M[i]);
    }
    int64_t kh = ks[h - 1];
    int64_t nb = (n + kh - 1) / kh;
    int levels = oracle_sparse_levels(nb);
    int32_t *T = rc == 0 ? (int32_t *)malloc((size_t)(nb * levels) * sizeof(int32_t)) : NULL;
    if (!T) rc = -1;
    if (rc == 0) {
        oracle_block_sparse_table(A, n, kh, T);
        for (int64_t i = 0; i < q; ++i) {
            int64_t wk = 0;
            if (!valid_query(n, l[i], r[i])) {
                out[i] = -1;
                if (work) work[i] = 0;
                continue;
            }
            int64_t bl = l[i] / kh, br = r[i] / kh;
            int32_t best;
            if (bl == br) {
                best = hlevel_part(A, M, ks, h, l[i], r[i], &wk);
            } else {
                best = hlevel_part(A, M, ks, h, l[i], (bl + 1) * kh - 1, &wk);
                if (br - bl >= 2) {
                    int t = ilog2_u64((uint64_t)(br - bl - 1));
                    best = lex_min(A, best, T[(int64_t)t * nb + bl + 1]);
                    best = lex_min(A, best, T[(int64_t)t * nb + br - ((int64_t)1 << t)]);
                    wk += 2;
                }
                best = lex_min(A, best, hlevel_part(A, M, ks, h, br * kh, r[i], &wk));
            }
            out[i] = best;
            if (work) work[i] = wk;
        }
    }
    for (int i = 0; i < 16; ++i) free(M[i]);
    free(T);
    return rc;
}
