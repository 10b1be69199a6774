/*
 * gf2_checks.c -- size-independent property checks of a PLE / RREF result.
 *
 * TEST INFRASTRUCTURE ONLY (same rules as gf2_oracle.c: used by tests/ and
 * bench.py's CPU leg, never by the product path, no code shared with it).
 *
 * At 32768^2 and 65536^2 the eager oracle takes minutes, so a result there is
 * verified by properties that together pin it uniquely:
 *
 *  1. check_ple_structure: E (the part of L\E on and right of the diagonal)
 *     is in row echelon form with pivot 1 at Q[i] (Section 2, Definition
 *     "Row Echelon Form"), Q strictly increasing, L has bits only in columns
 *     < rank (L's columns >= rank are the identity), P[i] >= i and P[i] = i
 *     past the rank (the swap vector of Section 1.2).
 *  2. check_freivalds_ple: P^T A X = L (E X) for 64 random vectors X at once
 *     (Freivalds' test; a wrong factorisation passes with probability
 *     <= 2^-64).  With 1., A = P L E holds (Definition "PLE Decomposition").
 *  3. check_pivot_rule: the row chosen at step p is the first row, in the
 *     order current at that step, whose reduced entry in column Q[p] is 1
 *     (Algorithm 1's column-wise search).  The rows passed over at step p are
 *     exactly the rows at positions [p, P[p]) then; their reduced entry in
 *     column Q[p] is the L coefficient they end up with for pivot p, so the
 *     rule is: L[final position of each such row][p] = 0.
 *     Given P, the factorisation with L's columns >= rank fixed to the
 *     identity is unique (L[:, :r] expresses P^T A in the basis E[:r]), and
 *     the column rule follows from 1.+2., so 1.-3. pin the whole output.
 *  4. check_rref: R is in reduced row echelon form with pivot columns Q
 *     (Definition "Reduced Row Echelon Form") and U R[:r] = E[:r] with
 *     U = E[:r, Q] (unit upper triangular), by the same random-vector test.
 *     Same row space as E (hence A) plus reduced echelon form is the unique
 *     RREF.
 *
 * Return value: 0 when the property holds, otherwise a positive code whose
 * low 4 bits name the failed check and whose high bits hold the row index.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define BIT(row, j) (((row)[(j) >> 6] >> ((j) & 63)) & 1ULL)
#define FAIL(code, row) ((int64_t)(code) | ((int64_t)(row) << 4))

static inline int64_t words_for(int64_t n) { return (n + 63) >> 6; }

static inline uint64_t splitmix64(uint64_t *x)
{
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Is bit j of row set, with columns < lo treated as zero. */
static inline uint64_t masked_word(const uint64_t *row, int64_t k, int64_t lo)
{
    uint64_t w = row[k];
    int64_t base = k << 6;
    if (lo > base) w = (lo - base >= 64) ? 0 : (w & (~0ULL << (lo - base)));
    return w;
}

/* Any set bit of row in columns [lo, hi)? */
static int any_bits(const uint64_t *row, int64_t lo, int64_t hi)
{
    for (int64_t k = lo >> 6; k < ((hi + 63) >> 6); ++k) {
        uint64_t w = row[k];
        int64_t base = k << 6;
        if (lo > base) w &= ~0ULL << (lo - base);
        if (hi < base + 64) w &= (1ULL << (hi - base)) - 1;
        if (w) return 1;
    }
    return 0;
}

int64_t check_ple_structure(const uint64_t *LE, int64_t m, int64_t n, int64_t ld,
                            const int64_t *P, const int64_t *Q, int64_t r)
{
    const int64_t W = words_for(n);
    int64_t qn = m < n ? m : n;
    if (r < 0 || r > qn) return FAIL(1, 0);
    for (int64_t i = 0; i < m; ++i) {
        if (P[i] < i || P[i] >= m) return FAIL(2, i);
        if (i >= r && P[i] != i) return FAIL(2, i);
    }
    for (int64_t i = 0; i < r; ++i) {
        if (Q[i] < 0 || Q[i] >= n || Q[i] < i) return FAIL(3, i);
        if (i > 0 && Q[i] <= Q[i - 1]) return FAIL(3, i);
    }
    for (int64_t i = r; i < qn; ++i)
        if (Q[i] != -1) return FAIL(3, i);
    int64_t ret = 0;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        const uint64_t *row = LE + i * ld;
        int64_t code = 0;
        if (n % 64 && (row[W - 1] >> (n % 64))) code = 4;          /* padding */
        else if (i < r) {
            if (any_bits(row, i, Q[i])) code = 5;                  /* zero in [i, Q[i]) */
            else if (!BIT(row, Q[i])) code = 6;                    /* pivot 1 */
        } else if (any_bits(row, r, n)) code = 7;                  /* past the rank */
        if (code) {
#pragma omp critical
            { if (!ret || (ret >> 4) > i) ret = FAIL(code, i); }
        }
    }
    return ret;
}

int64_t check_pivot_rule(const uint64_t *LE, int64_t m, int64_t ld,
                         const int64_t *P, int64_t r)
{
    int64_t *cur = (int64_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int64_t));
    int64_t *inv = (int64_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int64_t));
    if (!cur || !inv) { free(cur); free(inv); return FAIL(15, 0); }
    for (int64_t i = 0; i < m; ++i) cur[i] = i;
    for (int64_t p = 0; p < r; ++p) { int64_t t = cur[p]; cur[p] = cur[P[p]]; cur[P[p]] = t; }
    for (int64_t i = 0; i < m; ++i) inv[cur[i]] = i;       /* row id -> final position */
    for (int64_t i = 0; i < m; ++i) cur[i] = i;
    int64_t ret = 0;
    for (int64_t p = 0; p < r && !ret; ++p) {
        for (int64_t x = p; x < P[p]; ++x) {
            int64_t f = inv[cur[x]];
            if (f <= p || BIT(LE + f * ld, p)) { ret = FAIL(8, p); break; }
        }
        int64_t t = cur[p]; cur[p] = cur[P[p]]; cur[P[p]] = t;
    }
    free(cur); free(inv);
    return ret;
}

/* y[i] = XOR over set bits j >= lo_i of row i (columns < lim) of X[j]. */
static void project_rows(const uint64_t *M, int64_t m, int64_t ld, int64_t ncols,
                         const uint64_t *X, uint64_t *y, int diag_lo, int nthreads)
{
    const int64_t W = words_for(ncols);
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        const uint64_t *row = M + i * ld;
        uint64_t acc = 0;
        int64_t k0 = diag_lo ? (i >> 6) : 0;
        for (int64_t k = k0; k < W; ++k) {
            uint64_t w = diag_lo ? masked_word(row, k, i) : row[k];
            if (k == W - 1 && ncols % 64) w &= (1ULL << (ncols % 64)) - 1;
            while (w) {
                int b = __builtin_ctzll(w);
                acc ^= X[(k << 6) + b];
                w &= w - 1;
            }
        }
        y[i] = acc;
    }
}

int64_t check_freivalds_ple(const uint64_t *A0, int64_t ld0, const uint64_t *LE, int64_t ld,
                            int64_t m, int64_t n, const int64_t *P, int64_t r,
                            uint64_t seed, int nthreads)
{
    if (m <= 0 || n <= 0) return 0;
    uint64_t *X = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    uint64_t *y = (uint64_t *)malloc((size_t)m * sizeof(uint64_t));
    uint64_t *z = (uint64_t *)malloc((size_t)m * sizeof(uint64_t));
    uint64_t *w = (uint64_t *)malloc((size_t)m * sizeof(uint64_t));
    if (!X || !y || !z || !w) { free(X); free(y); free(z); free(w); return FAIL(15, 0); }
    uint64_t s = seed;
    for (int64_t j = 0; j < n; ++j) X[j] = splitmix64(&s);
    project_rows(A0, m, ld0, n, X, y, 0, nthreads);          /* y = A X */
    for (int64_t p = 0; p < r; ++p) { uint64_t t = y[p]; y[p] = y[P[p]]; y[P[p]] = t; }
    project_rows(LE, m, ld, n, X, z, 1, nthreads);           /* z = E X */
    /* w = L z: w[i] = z[i] ^ XOR_{p < min(i, r), L[i][p]} z[p] */
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        const uint64_t *row = LE + i * ld;
        int64_t lim = i < r ? i : r;
        uint64_t acc = z[i];
        for (int64_t k = 0; k < words_for(lim); ++k) {
            uint64_t bits = row[k];
            int64_t base = k << 6;
            if (lim - base < 64) bits &= (1ULL << (lim - base)) - 1;
            while (bits) {
                int b = __builtin_ctzll(bits);
                acc ^= z[base + b];
                bits &= bits - 1;
            }
        }
        w[i] = acc;
    }
    int64_t ret = 0;
    for (int64_t i = 0; i < m; ++i)
        if (w[i] != y[i]) { ret = FAIL(9, i); break; }
    free(X); free(y); free(z); free(w);
    return ret;
}

int64_t check_rref(const uint64_t *R, int64_t ldr, const uint64_t *LE, int64_t ld,
                   int64_t m, int64_t n, const int64_t *Q, int64_t r,
                   uint64_t seed, int nthreads)
{
    if (m <= 0 || n <= 0) return 0;
    const int64_t W = words_for(n);
    /* structure: row p has 1 at Q[p], zero left of it, zero at the other
     * pivot columns; rows >= r are zero */
    uint64_t *pm = (uint64_t *)calloc((size_t)W, sizeof(uint64_t));
    if (!pm) return FAIL(15, 0);
    for (int64_t q = 0; q < r; ++q) pm[Q[q] >> 6] |= 1ULL << (Q[q] & 63);
    int64_t sret = 0;
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        const uint64_t *row = R + i * ldr;
        int64_t code = 0;
        if (i >= r) {
            if (any_bits(row, 0, n)) code = 10;
        } else if (any_bits(row, 0, Q[i])) code = 11;
        else {
            for (int64_t k = 0; k < W && !code; ++k) {
                uint64_t want = (k == (Q[i] >> 6)) ? (1ULL << (Q[i] & 63)) : 0;
                if ((row[k] & pm[k]) != want) code = 12;
            }
        }
        if (code) {
#pragma omp critical
            { if (!sret || (sret >> 4) > i) sret = FAIL(code, i); }
        }
    }
    free(pm);
    if (sret) return sret;
    uint64_t *X = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    uint64_t *a = (uint64_t *)malloc((size_t)(r > 0 ? r : 1) * sizeof(uint64_t));
    uint64_t *b = (uint64_t *)malloc((size_t)(r > 0 ? r : 1) * sizeof(uint64_t));
    if (!X || !a || !b) { free(X); free(a); free(b); return FAIL(15, 0); }
    uint64_t s = seed;
    for (int64_t j = 0; j < n; ++j) X[j] = splitmix64(&s);
    project_rows(R, r, ldr, n, X, a, 0, nthreads);           /* a = R[:r] X */
    project_rows(LE, r, ld, n, X, b, 1, nthreads);           /* b = E[:r] X */
    int64_t ret = 0;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 64)
    for (int64_t p = 0; p < r; ++p) {
        const uint64_t *erow = LE + p * ld;
        uint64_t acc = a[p];
        for (int64_t q = p + 1; q < r; ++q)
            if (BIT(erow, Q[q])) acc ^= a[q];
        if (acc != b[p]) {
#pragma omp critical
            { if (!ret) ret = FAIL(13, p); }
        }
    }
    free(X); free(a); free(b);
    return ret;
}
