/*
 * gf2_oracle.c -- plain CPU oracle for dense GF(2) elimination.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file; only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg use it.  It shares no code with the CUDA path.
 *
 * Everything here is the plain definition, eager and unblocked, in the order
 * of the definitions it follows (Albrecht, Bard & Pernet, "Efficient Dense
 * Gaussian Elimination over the Finite Field with Two Elements"):
 *
 *   - PLE decomposition (Section 2, Definition "PLE Decomposition"): A = P L E,
 *     P a permutation stored LAPACK-style as a swap vector (Section 1.2, the
 *     5x5 example P = [0,2,2,4,4]), L unit lower triangular m x m, E in row
 *     echelon form.  Pivots are searched column-wise: the leftmost column that
 *     still has a nonzero, and in it the first row in the current (already
 *     swapped) order (Section 3.1, Algorithm 1 "PartialPle"; Algorithm 2
 *     "Ensures": Q_i is the column of the i-th pivot).
 *   - The output overwrites A with the space-sharing form L\E (Section 1.2):
 *     a_ij = l_ij for i > j, a_ij = e_ij otherwise.  L's columns >= rank are
 *     the identity, so only columns < rank carry L bits.
 *   - RREF (Section 2, Definition "Reduced Row Echelon Form"), recovered from
 *     E by clearing every pivot column above its pivot (Section 5 computes
 *     the RREF "from the PLE form"; the method is not described, so this is
 *     the textbook back-substitution).
 *   - Products over GF(2): C[i] = XOR over l with A[i][l] = 1 of B[l].
 *   - Solving A X = B through the PLE decomposition (Section 1 names solving
 *     as the use of the decomposition; the conventions -- free variables 0,
 *     status codes -- are this library's).
 *
 * Bit layout: row-major, ld uint64 words per row, column j = bit (j % 64) of
 * word j / 64.  Padding bits (columns >= n) are zero on input and output.
 *
 * Multithreading: OpenMP over independent rows inside one pivot step; the
 * result does not depend on the thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define BIT(row, j) (((row)[(j) >> 6] >> ((j) & 63)) & 1ULL)

static inline int64_t words_for(int64_t n) { return (n + 63) >> 6; }

static void swap_rows(uint64_t *X, int64_t ld, int64_t a, int64_t b, int64_t w)
{
    if (a == b) return;
    uint64_t *ra = X + a * ld, *rb = X + b * ld;
    for (int64_t k = 0; k < w; ++k) { uint64_t t = ra[k]; ra[k] = rb[k]; rb[k] = t; }
}

/*
 * Eager Gaussian elimination with the PLE pivot rule.
 *
 * E (in place, m x n, ld words): on return rows 0..r-1 hold E's nonzero rows
 * (echelon, pivot 1 at Q[i]); rows >= r are zero in columns < npiv.
 * L (m x lw words, may be NULL): L[t] bit p = 1 iff pivot row p was added to
 * the row now at position t.  Rows of L move with the rows of E.
 * Only columns < npiv are eligible as pivot columns; elimination still acts
 * on the full row (this is what the augmented [A | B] solve needs).
 * At most max_pivots pivots are taken (max_pivots < 0: no limit); a limited
 * run is a prefix of the full elimination, used to time a bounded sample.
 */
static int64_t eliminate(uint64_t *E, int64_t m, int64_t n, int64_t ld, int64_t npiv,
                         int64_t max_pivots, int64_t *P, int64_t *Q,
                         uint64_t *L, int64_t lw, int nthreads)
{
    const int64_t W = words_for(n);
    int64_t r = 0;
    if (max_pivots < 0) max_pivots = m;
    for (int64_t i = 0; i < m; ++i) P[i] = i;
    for (int64_t j = 0; j < npiv && r < m && r < max_pivots; ++j) {
        int64_t piv = -1;
        for (int64_t i = r; i < m; ++i) {
            if (BIT(E + i * ld, j)) { piv = i; break; }
        }
        if (piv < 0) continue;                  /* no pivot in column j */
        P[r] = piv;
        Q[r] = j;
        swap_rows(E, ld, r, piv, W);
        if (L) swap_rows(L, lw, r, piv, lw);
        const uint64_t *prow = E + r * ld;
        const int64_t w0 = j >> 6;
        const int64_t pr = r;
#pragma omp parallel for num_threads(nthreads) schedule(static)
        for (int64_t t = pr + 1; t < m; ++t) {
            uint64_t *row = E + t * ld;
            if (BIT(row, j)) {
                for (int64_t k = w0; k < W; ++k) row[k] ^= prow[k];
                if (L) L[t * lw + (pr >> 6)] |= 1ULL << (pr & 63);
            }
        }
        ++r;
    }
    return r;
}

/*
 * PLE decomposition, output in the space-sharing form L\E (Section 1.2).
 * P: int64[m] swap vector (row i was swapped with P[i] at step i; P[i] = i
 * for i >= rank).  Q: int64[min(m, npiv)], Q[i] = column of the i-th pivot,
 * -1 past the rank.  Returns the rank, or -1 if memory runs out.
 */
int64_t oracle_ple(uint64_t *A, int64_t m, int64_t n, int64_t ld, int64_t npiv,
                   int64_t max_pivots, int64_t *P, int64_t *Q, int nthreads)
{
    if (m <= 0 || n <= 0) { for (int64_t i = 0; i < m; ++i) P[i] = i; return 0; }
    if (npiv > n || npiv < 0) npiv = n;
    int64_t qn = m < npiv ? m : npiv;
    int64_t lcols = qn;
    if (max_pivots >= 0 && max_pivots < lcols) lcols = max_pivots;
    int64_t lw = words_for(lcols > 0 ? lcols : 1);
    uint64_t *L = (uint64_t *)calloc((size_t)(m * lw), sizeof(uint64_t));
    if (!L) return -1;
    for (int64_t i = 0; i < qn; ++i) Q[i] = -1;
    int64_t r = eliminate(A, m, n, ld, npiv, max_pivots, P, Q, L, lw, nthreads);
    /* Compose L\E: E is zero strictly left of each row's diagonal, and L has
     * bits only in columns p < min(i, r); OR them in. */
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int64_t i = 0; i < m; ++i)
        for (int64_t k = 0; k < lw; ++k) A[i * ld + k] |= L[i * lw + k];
    free(L);
    return r;
}

/*
 * Reduced row echelon form of A in place (rows >= rank become zero).
 * Q: int64[min(m, n)] pivot columns, -1 past the rank.  Returns the rank.
 */
int64_t oracle_rref(uint64_t *A, int64_t m, int64_t n, int64_t ld, int64_t *Q, int nthreads)
{
    if (m <= 0 || n <= 0) return 0;
    const int64_t W = words_for(n);
    int64_t qn = m < n ? m : n;
    int64_t *P = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    if (!P) return -1;
    for (int64_t i = 0; i < qn; ++i) Q[i] = -1;
    int64_t r = eliminate(A, m, n, ld, n, -1, P, Q, NULL, 0, nthreads);
    free(P);
    /* Back-substitution: clear column Q[p] in every row above p, last pivot
     * first, so each row added is already reduced against later pivots. */
    for (int64_t p = r - 1; p >= 0; --p) {
        const int64_t j = Q[p];
        const uint64_t *prow = A + p * ld;
        const int64_t w0 = j >> 6;
#pragma omp parallel for num_threads(nthreads) schedule(static)
        for (int64_t q = 0; q < p; ++q) {
            uint64_t *row = A + q * ld;
            if (BIT(row, j))
                for (int64_t k = w0; k < W; ++k) row[k] ^= prow[k];
        }
    }
    for (int64_t i = r; i < m; ++i) memset(A + i * ld, 0, (size_t)W * sizeof(uint64_t));
    return r;
}

/*
 * C = A * B (accumulate = 0) or C ^= A * B (accumulate != 0) over GF(2).
 * A: m x k (lda), B: k x n (ldb), C: m x n (ldc).
 */
void oracle_mul(uint64_t *C, int64_t ldc, const uint64_t *A, int64_t lda,
                const uint64_t *B, int64_t ldb, int64_t m, int64_t k, int64_t n,
                int accumulate, int nthreads)
{
    const int64_t W = words_for(n);
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        uint64_t *crow = C + i * ldc;
        if (!accumulate) memset(crow, 0, (size_t)W * sizeof(uint64_t));
        const uint64_t *arow = A + i * lda;
        for (int64_t l = 0; l < k; ++l) {
            if (BIT(arow, l)) {
                const uint64_t *brow = B + l * ldb;
                for (int64_t w = 0; w < W; ++w) crow[w] ^= brow[w];
            }
        }
    }
}

/*
 * Solve A X = B for square A (n x n) through PLE.
 * A is overwritten with L\E.  B (n x nrhs, ldb) is overwritten with X when
 * the system is consistent: X[Q[p]] from back-substitution on E's pivot
 * columns, X[non-pivot columns] = 0.  Returns 0 (unique solution, rank n),
 * 1 (consistent, rank < n; free variables set to 0), 2 (inconsistent: some
 * row >= rank of L^-1 P^T B is nonzero; B then holds that transformed
 * right-hand side).  *rank_out receives the rank.  -1 on allocation failure.
 */
int oracle_solve(uint64_t *A, int64_t n, int64_t lda, uint64_t *B, int64_t nrhs,
                 int64_t ldb, int64_t *rank_out, int nthreads)
{
    if (n <= 0) { *rank_out = 0; return 0; }
    const int64_t bw = words_for(nrhs > 0 ? nrhs : 1);
    const int64_t lw = words_for(n);
    int64_t *P = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *Q = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    uint64_t *L = (uint64_t *)calloc((size_t)(n * lw), sizeof(uint64_t));
    uint64_t *X = (uint64_t *)calloc((size_t)(n * bw), sizeof(uint64_t));
    if (!P || !Q || !L || !X) { free(P); free(Q); free(L); free(X); return -1; }
    int64_t r = eliminate(A, n, n, lda, n, -1, P, Q, L, lw, nthreads);
    *rank_out = r;
    /* Y = P^T B: the swaps in the order they were made. */
    for (int64_t p = 0; p < r; ++p) swap_rows(B, ldb, p, P[p], bw);
    /* Y = L^-1 Y, forward substitution row by row. */
    for (int64_t i = 1; i < n; ++i) {
        uint64_t *yi = B + i * ldb;
        int64_t lim = i < r ? i : r;
        for (int64_t p = 0; p < lim; ++p)
            if (BIT(L + i * lw, p))
                for (int64_t w = 0; w < bw; ++w) yi[w] ^= B[p * ldb + w];
    }
    int status = (r == n) ? 0 : 1;
    for (int64_t i = r; i < n && status != 2; ++i)
        for (int64_t w = 0; w < bw; ++w)
            if (B[i * ldb + w]) { status = 2; break; }
    if (status != 2) {
        /* Back-substitution on E's pivot columns, last pivot first. */
        for (int64_t p = r - 1; p >= 0; --p) {
            uint64_t *xp = X + Q[p] * bw;
            for (int64_t w = 0; w < bw; ++w) xp[w] = B[p * ldb + w];
            for (int64_t q = p + 1; q < r; ++q)
                if (BIT(A + p * lda, Q[q]))
                    for (int64_t w = 0; w < bw; ++w) xp[w] ^= X[Q[q] * bw + w];
        }
        for (int64_t i = 0; i < n; ++i)
            for (int64_t w = 0; w < bw; ++w) B[i * ldb + w] = X[i * bw + w];
    }
    /* A <- L\E */
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = 0; k < lw; ++k) A[i * lda + k] |= L[i * lw + k];
    free(P); free(Q); free(L); free(X);
    return status;
}
