/*
 * oracle.c -- the plain, slow CPU reference for exact Gauss-Jordan elimination
 * over the prime field Z/pZ.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call,
 * link or load this file: only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * What it computes (paper section 3.2, "Gaussian elimination on GPUs"):
 * partially pivoted row reduction to the reduced row-echelon form (RREF),
 * looping over the columns one at a time ("Looping"), searching the current
 * column for a usable pivot ("Pivoting": over a finite field any nonzero
 * entry will do, and the RREF does not depend on which one is taken -- this
 * oracle takes the lowest-index nonzero row), swapping it into place,
 * scaling the pivot row so the head becomes 1 ("Conditional Rescale"), and
 * subtracting multiples of the pivot row from EVERY other row, above and
 * below, so the pivot column becomes a unit vector ("Row reduce"); the row
 * counter advances only when the head was nonzero ("Increment counters").
 * The output keeps the input shape, zero rows at the bottom (section 2.3).
 *
 * Arithmetic: entries are canonical residues in [0, p), p an odd prime below
 * 2^31.  Every product is formed in uint64_t (< 2^62) and reduced with the C
 * '%' operator -- no Barrett, Montgomery, Shoup or limb tricks.  Inverses are
 * Fermat's h^(p-2) mod p by square-and-multiply.  The functions at the end of
 * the file (oracle_rref64, oracle_solve64, oracle_inverse64) repeat the
 * elimination for uint64 residues and primes below 2^64, with products in
 * unsigned __int128; they are pinned in tests/test_oracle64_pins.py.
 *
 * Threads: the row updates of one pivot step are independent of one another;
 * with nthreads > 1 each thread owns a contiguous range of rows and the
 * threads meet at a barrier after the pivot step and after the updates.  The
 * arithmetic is identical for every thread count.
 *
 * Parity pins: every function here is pinned in tests/test_oracle_pins.py to
 * facts fixed by the mathematics (RREF of a matrix built from a known RREF,
 * brute-force rank over all minors, brute-force null spaces and solution
 * sets for tiny p, closed-form Vandermonde and L*D*U determinants,
 * polynomial interpolation).
 */
#define _POSIX_C_SOURCE 200809L
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* h^e mod p by binary exponentiation; uint64 products of residues < 2^62. */
static uint64_t oracle_powmod(uint64_t h, uint64_t e, uint64_t p) {
    uint64_t result = 1 % p;
    h %= p;
    while (e) {
        if (e & 1) result = (result * h) % p;
        h = (h * h) % p;
        e >>= 1;
    }
    return result;
}

/* Fermat's little theorem: h^(p-1) = 1 for h != 0, so h^(p-2) = 1/h. */
uint32_t oracle_inverse(uint32_t h, uint32_t p) {
    return (uint32_t)oracle_powmod(h, (uint64_t)p - 2, p);
}

typedef struct {
    uint32_t *A;
    int64_t m, n, ld;
    uint64_t p;
    int64_t col_limit;    /* pivots are searched in columns [0, col_limit) */
    int64_t max_pivots;   /* stop after this many pivots (< 0: no limit) */
    int nthreads;
    pthread_barrier_t bar;
    /* state written by thread 0 between barriers */
    int64_t r;            /* current rank = index of the next pivot row */
    int64_t c;            /* current column */
    int found;            /* the current column has a nonzero head */
    int done;
    int32_t *pivots;
    uint64_t det_sign_neg; /* parity of row swaps */
    uint64_t det_prod;     /* product of the heads before scaling */
} oracle_ctx;

typedef struct { oracle_ctx *C; int tid; } oracle_arg;

/* Pivot step for column c (section 3.2, "Pivoting" and "Conditional
 * Rescale"): find the lowest row q >= r with A[q][c] != 0, swap rows q and r,
 * multiply row r by the inverse of its head. */
static void oracle_pivot_step(oracle_ctx *C) {
    const int64_t n = C->n, ld = C->ld, c = C->c, r = C->r;
    const uint64_t p = C->p;
    uint32_t *A = C->A;
    int64_t q = -1;
    for (int64_t i = r; i < C->m; i++) {
        if (A[i * ld + c] != 0) { q = i; break; }
    }
    if (q < 0) { C->found = 0; return; }
    C->found = 1;
    if (q != r) {
        for (int64_t j = 0; j < n; j++) {
            uint32_t t = A[q * ld + j];
            A[q * ld + j] = A[r * ld + j];
            A[r * ld + j] = t;
        }
        C->det_sign_neg ^= 1;
    }
    uint64_t h = A[r * ld + c];
    C->det_prod = (C->det_prod * h) % p;
    uint64_t hinv = oracle_inverse((uint32_t)h, (uint32_t)p);
    for (int64_t j = c; j < n; j++)
        A[r * ld + j] = (uint32_t)(((uint64_t)A[r * ld + j] * hinv) % p);
}

/* Row update for rows [lo, hi) (section 3.2, "Row reduce"): every row i other
 * than the pivot row with a nonzero entry f in the pivot column becomes
 * row_i - f * row_r; columns left of c are zero in row r and are skipped. */
static void oracle_update_rows(oracle_ctx *C, int64_t lo, int64_t hi) {
    const int64_t n = C->n, ld = C->ld, c = C->c, r = C->r;
    const uint64_t p = C->p;
    uint32_t *A = C->A;
    const uint32_t *prow = A + r * ld;
    for (int64_t i = lo; i < hi; i++) {
        if (i == r) continue;
        uint32_t *row = A + i * ld;
        uint64_t f = row[c];
        if (f == 0) continue;
        uint64_t negf = p - f;
        for (int64_t j = c; j < n; j++)
            row[j] = (uint32_t)(((uint64_t)row[j] + negf * (uint64_t)prow[j]) % p);
    }
}

static void *oracle_worker(void *argp) {
    oracle_arg *arg = (oracle_arg *)argp;
    oracle_ctx *C = arg->C;
    const int tid = arg->tid, T = C->nthreads;
    const int64_t m = C->m;
    const int64_t lo = (m * tid) / T, hi = (m * (tid + 1)) / T;
    for (;;) {
        if (tid == 0) {
            if (C->c >= C->col_limit || C->r >= m ||
                (C->max_pivots >= 0 && C->r >= C->max_pivots)) {
                C->done = 1;
            } else {
                oracle_pivot_step(C);
            }
        }
        pthread_barrier_wait(&C->bar);
        if (C->done) break;
        if (C->found) oracle_update_rows(C, lo, hi);
        pthread_barrier_wait(&C->bar);
        if (tid == 0) {   /* section 3.2, "Increment counters" */
            if (C->found) { C->pivots[C->r] = (int32_t)C->c; C->r++; }
            C->c++;
        }
    }
    return NULL;
}

/*
 * In-place RREF of the m x n row-major matrix A (leading dimension ld).
 * Pivots are searched in columns [0, col_limit) only; the remaining columns
 * are carried along (used by oracle_solve).  max_pivots < 0 means run to the
 * end; otherwise the elimination stops once that many pivots were taken (a
 * bounded sample for timing).
 * Outputs: *rank, pivots[0..rank) (the rest of pivots[0..min(m,n)) is set to
 * -1), *det_out = (-1)^swaps * product of the heads before scaling, which is
 * det(A) when A is square, col_limit == n and the rank is n (zero if the rank
 * is short).
 * Returns 0, or -1 for bad arguments.
 */
int oracle_rref(uint32_t *A, int64_t m, int64_t n, int64_t ld, uint32_t p,
                int64_t col_limit, int64_t max_pivots, int nthreads,
                int32_t *rank, int32_t *pivots, uint32_t *det_out) {
    if (m < 0 || n < 0 || ld < n || p < 2 || col_limit < 0 || col_limit > n)
        return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    int64_t mn = m < n ? m : n;
    for (int64_t i = 0; i < mn; i++) pivots[i] = -1;
    oracle_ctx C;
    memset(&C, 0, sizeof C);
    C.A = A; C.m = m; C.n = n; C.ld = ld; C.p = p;
    C.col_limit = col_limit; C.max_pivots = max_pivots;
    C.nthreads = nthreads; C.pivots = pivots;
    C.det_prod = 1 % p;
    pthread_barrier_init(&C.bar, NULL, (unsigned)nthreads);
    oracle_arg args[256];
    pthread_t th[256];
    for (int t = 0; t < nthreads; t++) { args[t].C = &C; args[t].tid = t; }
    for (int t = 1; t < nthreads; t++) pthread_create(&th[t], NULL, oracle_worker, &args[t]);
    oracle_worker(&args[0]);
    for (int t = 1; t < nthreads; t++) pthread_join(th[t], NULL);
    pthread_barrier_destroy(&C.bar);
    *rank = (int32_t)C.r;
    if (det_out) {
        uint64_t d = C.det_prod;
        if (C.r < mn || m != n) d = 0;
        if (C.det_sign_neg && d) d = p - d;
        *det_out = (uint32_t)d;
    }
    return 0;
}

/*
 * Solve A X = B over Z/pZ (section 5.2, "Solving linear systems"): reduce
 * the augmented matrix M = [A | B] (m x (nA + k), leading dimension ld,
 * overwritten) with pivots restricted to A's columns.  Right-hand side j is
 * consistent iff rank(A) = rank(A | b_j), i.e. iff column j of the reduced B
 * vanishes in every row at or below the rank.  The particular solution sets
 * every free variable to zero: X[pivots[t]][j] = reduced B[t][j], other rows 0.
 * X is nA x k with leading dimension ldx; inconsistent columns of X are 0.
 */
int oracle_solve(uint32_t *M, int64_t m, int64_t nA, int64_t k, int64_t ld,
                 uint32_t p, int nthreads, uint32_t *X, int64_t ldx,
                 uint8_t *consistent, int32_t *rank, int32_t *pivots) {
    if (k < 0 || ldx < k) return -1;
    int rc = oracle_rref(M, m, nA + k, ld, p, nA, -1, nthreads, rank, pivots, NULL);
    if (rc) return rc;
    const int64_t r = *rank;
    for (int64_t i = 0; i < nA; i++)
        for (int64_t j = 0; j < k; j++) X[i * ldx + j] = 0;
    for (int64_t j = 0; j < k; j++) {
        int ok = 1;
        for (int64_t i = r; i < m; i++)
            if (M[i * ld + nA + j] != 0) { ok = 0; break; }
        consistent[j] = (uint8_t)ok;
        if (!ok) continue;
        for (int64_t t = 0; t < r; t++)
            X[(int64_t)pivots[t] * ldx + j] = M[t * ld + nA + j];
    }
    return 0;
}

/*
 * Matrix construction of paper section 3.3 ("Building linear systems on
 * GPUs") and section 2.3 (cuda_load_matrix): each row r is one sampling
 * point given by its basis-variable values bases[r][0..n_basis), each column
 * c one monomial given by d indices into those values, and
 *     A[r][c] = prod_{t < d} bases[r][lindices[c][t]]  mod p.
 * The product is taken left to right, reducing after every factor.
 * lindices is n_cols x d, row-major.  Returns -1 for an index out of range.
 */
int oracle_load_matrix(const uint32_t *bases, int64_t n_rows, int64_t n_basis, int64_t ldb,
                       const int32_t *lindices, int64_t n_cols, int64_t d, uint32_t p,
                       uint32_t *A, int64_t lda) {
    if (n_rows < 0 || n_cols < 0 || d < 0 || ldb < n_basis || lda < n_cols || p < 2) return -1;
    for (int64_t c = 0; c < n_cols; c++)
        for (int64_t t = 0; t < d; t++)
            if (lindices[c * d + t] < 0 || lindices[c * d + t] >= n_basis) return -1;
    for (int64_t r = 0; r < n_rows; r++) {
        for (int64_t c = 0; c < n_cols; c++) {
            uint64_t v = 1 % p;
            for (int64_t t = 0; t < d; t++)
                v = (v * (uint64_t)bases[r * ldb + lindices[c * d + t]]) % p;
            A[r * lda + c] = (uint32_t)v;
        }
    }
    return 0;
}

/*
 * Plain matrix product over Z/pZ: C = A B mod p, A m x K, B K x n, all
 * row-major with canonical residues.  Each product is reduced before it is
 * added (uint64 '%').  Used to state the paper's identities A = C R (rank
 * factorisation, section 5.1) and A K = 0 (null space, section 5.1), and to
 * expand a template of polynomial entries at many points (section 3.3).
 */
int oracle_matmul(const uint32_t *A, int64_t m, int64_t K, int64_t lda,
                  const uint32_t *B, int64_t n, int64_t ldb, uint32_t p,
                  uint32_t *C, int64_t ldc) {
    if (m < 0 || K < 0 || n < 0 || lda < K || ldb < n || ldc < n || p < 2) return -1;
    for (int64_t i = 0; i < m; i++) {
        for (int64_t j = 0; j < n; j++) {
            uint64_t s = 0;
            for (int64_t k = 0; k < K; k++)
                s = (s + ((uint64_t)A[i * lda + k] * (uint64_t)B[k * ldb + j]) % p) % p;
            C[i * ldc + j] = (uint32_t)s;
        }
    }
    return 0;
}

/*
 * LUP factorisation P A = L U (paper section 6, "Conclusions and Outlook",
 * names an LUP factorisation as the option to add beside the rank
 * decomposition; the paper does not define it further, so this is the
 * reading the library implements).  The elimination is the column loop of
 * section 3.2 with two changes: only the rows that are not yet pivots are
 * reduced (no "Row reduce" of the rows above, no rescaling of the pivot row),
 * and the multiplier f / h of every reduced row is kept in L.  The pivot of
 * column c is the lowest-index row, in the ORIGINAL order, among the rows that
 * are not yet pivots and have a nonzero entry in column c ("Pivoting": any
 * nonzero entry will do; this rule makes P, L and U unique).  With r the rank:
 *   perm[t] (t < r)   the pivot row of the t-th pivot column pivots[t];
 *   perm[r..m-1]      the other rows in increasing order;
 *   U (m x n)         row t < r is row perm[t] after the elimination (zero
 *                     left of pivots[t], head U[t][pivots[t]] != 0); rows
 *                     r..m-1 are zero;
 *   L (m x min(m,n))  the first min(m,n) columns of the m x m unit lower
 *                     triangular factor: L[i][i] = 1, L[i][t] for i > t, t < r
 *                     is the multiplier row perm[i] took for pivot t, and
 *                     column t >= r is the unit vector e_t.
 * Row i of P A is row perm[i] of A.  Every product is reduced with '%'.
 * The work matrix W (m x n, leading dimension n) and Lo (m x min(m,n)) are
 * caller-provided scratch.  Returns 0, or -1 for bad arguments.
 */
int oracle_lup(const uint32_t *A, int64_t m, int64_t n, int64_t ld, uint32_t p,
               uint32_t *L, int64_t ldl, uint32_t *U, int64_t ldu,
               int32_t *perm, int32_t *rank, int32_t *pivots,
               uint32_t *W, uint32_t *Lo, uint8_t *is_pivot) {
    if (m < 0 || n < 0 || ld < n || p < 2) return -1;
    const int64_t mn = m < n ? m : n;
    if (ldl < mn || ldu < n) return -1;
    for (int64_t i = 0; i < m; i++) {
        is_pivot[i] = 0;
        for (int64_t j = 0; j < n; j++) W[i * n + j] = A[i * ld + j];
        for (int64_t t = 0; t < mn; t++) Lo[i * mn + t] = 0;
    }
    for (int64_t t = 0; t < mn; t++) pivots[t] = -1;
    int64_t r = 0;
    for (int64_t c = 0; c < n && r < m; c++) {
        int64_t q = -1;
        for (int64_t i = 0; i < m; i++)
            if (!is_pivot[i] && W[i * n + c] != 0) { q = i; break; }
        if (q < 0) continue;
        const uint64_t hinv = oracle_inverse(W[q * n + c], p);
        for (int64_t i = 0; i < m; i++) {
            if (is_pivot[i] || i == q) continue;
            const uint64_t f = W[i * n + c];
            if (f == 0) continue;
            const uint64_t l = (f * hinv) % p;
            Lo[i * mn + r] = (uint32_t)l;
            const uint64_t negl = p - l;
            for (int64_t j = c; j < n; j++)
                W[i * n + j] = (uint32_t)(((uint64_t)W[i * n + j] + negl * (uint64_t)W[q * n + j]) % p);
        }
        is_pivot[q] = 1;
        perm[r] = (int32_t)q;
        pivots[r] = (int32_t)c;
        r++;
    }
    *rank = (int32_t)r;
    int64_t t = r;
    for (int64_t i = 0; i < m; i++)
        if (!is_pivot[i]) perm[t++] = (int32_t)i;
    for (int64_t i = 0; i < m; i++) {
        for (int64_t s = 0; s < mn; s++) {
            uint32_t v;
            if (s == i) v = 1;
            else if (s < i && s < r) v = Lo[(int64_t)perm[i] * mn + s];
            else v = 0;
            L[i * ldl + s] = v;
        }
        for (int64_t j = 0; j < n; j++) U[i * ldu + j] = i < r ? W[(int64_t)perm[i] * n + j] : 0;
    }
    return 0;
}

/* ===========================================================================
 * 64-bit residues.  Section 2.3 ("Basic Usage"): residues are held as uint64
 * when p does not fit 32 bits, for primes up to 2^64 - 1 (and section 3.4,
 * "Optimisations", reads them two at a time as ulonglong2).  The elimination
 * below is the same column loop as oracle_rref (section 3.2: Looping,
 * Pivoting with the lowest-index nonzero row, Conditional Rescale by the
 * Fermat inverse, Row reduce over every other row, Increment counters); only
 * the number type differs.  Every product is formed in unsigned __int128
 * (below 2^128) and reduced with the C '%' operator.
 * ======================================================================== */

typedef unsigned __int128 o_u128;

static uint64_t o64_mul(uint64_t a, uint64_t b, uint64_t p) {
    return (uint64_t)(((o_u128)a * (o_u128)b) % p);
}

static uint64_t o64_pow(uint64_t h, uint64_t e, uint64_t p) {
    uint64_t acc = 1 % p;
    h %= p;
    for (; e; e >>= 1) {
        if (e & 1) acc = o64_mul(acc, h, p);
        h = o64_mul(h, h, p);
    }
    return acc;
}

/* 1/h mod p = h^(p-2) mod p (Fermat), h != 0. */
uint64_t oracle_inverse64(uint64_t h, uint64_t p) { return o64_pow(h, p - 2, p); }

typedef struct {
    uint64_t *A;
    int64_t m, n, ld;
    uint64_t p;
    int64_t col_limit;
    int nthreads;
    pthread_barrier_t bar;
    int64_t rank_now, col_now;   /* written by thread 0 between barriers */
    int have_pivot, finished;
    int32_t *pivots;
} o64_ctx;

typedef struct { o64_ctx *C; int tid; } o64_arg;

/* Column col_now: the lowest row at or below rank_now with a nonzero entry
 * becomes the pivot row; it is swapped into row rank_now and scaled by the
 * inverse of its head. */
static void o64_pivot(o64_ctx *C) {
    const int64_t ld = C->ld, c = C->col_now, r = C->rank_now;
    uint64_t *A = C->A;
    int64_t q = r;
    while (q < C->m && A[q * ld + c] == 0) q++;
    C->have_pivot = q < C->m;
    if (!C->have_pivot) return;
    for (int64_t j = 0; q != r && j < C->n; j++) {
        uint64_t t = A[q * ld + j];
        A[q * ld + j] = A[r * ld + j];
        A[r * ld + j] = t;
    }
    uint64_t hinv = oracle_inverse64(A[r * ld + c], C->p);
    for (int64_t j = c; j < C->n; j++) A[r * ld + j] = o64_mul(A[r * ld + j], hinv, C->p);
}

/* Rows [lo, hi) other than the pivot row: row_i -= row_i[c] * pivot_row,
 * written as row_i + (p - f) * pivot_row so every term stays unsigned. */
static void o64_reduce_rows(o64_ctx *C, int64_t lo, int64_t hi) {
    const int64_t ld = C->ld, c = C->col_now, prow = C->rank_now;
    const uint64_t p = C->p;
    uint64_t *A = C->A;
    for (int64_t i = lo; i < hi; i++) {
        uint64_t f = A[i * ld + c];
        if (i == prow || f == 0) continue;
        uint64_t minus_f = p - f;
        for (int64_t j = c; j < C->n; j++) {
            o_u128 v = (o_u128)A[i * ld + j] + (o_u128)minus_f * A[prow * ld + j];
            A[i * ld + j] = (uint64_t)(v % p);
        }
    }
}

static void *o64_worker(void *argp) {
    o64_arg *arg = (o64_arg *)argp;
    o64_ctx *C = arg->C;
    const int64_t lo = (C->m * arg->tid) / C->nthreads, hi = (C->m * (arg->tid + 1)) / C->nthreads;
    for (;;) {
        if (arg->tid == 0) {
            C->finished = C->col_now >= C->col_limit || C->rank_now >= C->m;
            if (!C->finished) o64_pivot(C);
        }
        pthread_barrier_wait(&C->bar);
        if (C->finished) break;
        if (C->have_pivot) o64_reduce_rows(C, lo, hi);
        pthread_barrier_wait(&C->bar);
        if (arg->tid == 0) {
            if (C->have_pivot) C->pivots[C->rank_now++] = (int32_t)C->col_now;
            C->col_now++;
        }
    }
    return NULL;
}

/* In-place RREF of the m x n uint64 matrix A (leading dimension ld) over
 * Z/pZ, 3 <= p < 2^64 prime, pivots searched in columns [0, col_limit).
 * pivots[0..min(m,n)) gets the pivot columns, -1 after the rank.
 * Returns 0, or -1 for bad arguments. */
int oracle_rref64(uint64_t *A, int64_t m, int64_t n, int64_t ld, uint64_t p, int64_t col_limit,
                  int nthreads, int32_t *rank, int32_t *pivots) {
    if (m < 0 || n < 0 || ld < n || p < 3 || col_limit < 0 || col_limit > n) return -1;
    nthreads = nthreads < 1 ? 1 : (nthreads > 256 ? 256 : nthreads);
    for (int64_t i = 0; i < (m < n ? m : n); i++) pivots[i] = -1;
    o64_ctx C;
    memset(&C, 0, sizeof C);
    C.A = A; C.m = m; C.n = n; C.ld = ld; C.p = p; C.col_limit = col_limit;
    C.nthreads = nthreads; C.pivots = pivots;
    pthread_barrier_init(&C.bar, NULL, (unsigned)nthreads);
    o64_arg args[256];
    pthread_t th[256];
    for (int t = 0; t < nthreads; t++) { args[t].C = &C; args[t].tid = t; }
    for (int t = 1; t < nthreads; t++) pthread_create(&th[t], NULL, o64_worker, &args[t]);
    o64_worker(&args[0]);
    for (int t = 1; t < nthreads; t++) pthread_join(th[t], NULL);
    pthread_barrier_destroy(&C.bar);
    *rank = (int32_t)C.rank_now;
    return 0;
}

/* Section 5.2 with uint64 residues: reduce M = [A | B] with pivots in A's
 * nA columns; column j of B is consistent iff its reduced entries vanish at
 * and below the rank; X[pivots[t]][j] = reduced B[t][j], free variables and
 * inconsistent columns zero. */
int oracle_solve64(uint64_t *M, int64_t m, int64_t nA, int64_t k, int64_t ld, uint64_t p, int nthreads,
                   uint64_t *X, int64_t ldx, uint8_t *consistent, int32_t *rank, int32_t *pivots) {
    if (k < 0 || ldx < k) return -1;
    if (oracle_rref64(M, m, nA + k, ld, p, nA, nthreads, rank, pivots)) return -1;
    for (int64_t i = 0; i < nA * ldx; i++) X[i] = 0;
    for (int64_t j = 0; j < k; j++) {
        int64_t i = *rank;
        while (i < m && M[i * ld + nA + j] == 0) i++;
        consistent[j] = (uint8_t)(i == m);
        for (int64_t t = 0; consistent[j] && t < *rank; t++)
            X[pivots[t] * ldx + j] = M[t * ld + nA + j];
    }
    return 0;
}
