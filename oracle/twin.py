"""Second, independent PLE implementation on unpacked 0/1 arrays.

TEST INFRASTRUCTURE ONLY.  Pure Python loops, for small matrices (m, n up to
a few hundred).  It shares nothing with ``gf2_oracle.c`` except the problem
statement, and it is organised differently on purpose:

* it works on unpacked ``uint8`` arrays with explicit column indices, so it
  is independent of the packed bit order;
* it is *lazy* (left-looking), as Algorithm 1 ("PartialPle", Section 3.1)
  is: a row is brought up to date with the pivots found so far only at the
  moment its entry in the current column has to be inspected, and the
  remaining rows are caught up at the end.  The C oracle is eager
  (right-looking).  Both must find the same pivots (column-wise search:
  leftmost column with a nonzero, first row in the current order; rows are
  exchanged by swaps recorded LAPACK-style, Section 1.2), so agreement pins
  the reading of the pivot rule and of the swap vector.

Instead of Algorithm 1's per-pivot s-array this keeps, per row, the number of
pivots it has already been updated against (the same bookkeeping seen from
the row side).  L is kept as an explicit m x m matrix and E separately; the
space-sharing form L\\E of Section 1.2 is formed by ``compact``.
"""
from __future__ import annotations

import numpy as np


def ple(A01: np.ndarray):
    """Lazy PLE of an unpacked m x n 0/1 matrix.

    Returns ``(r, P, Q, L, E)``: rank, swap vector (length m), pivot columns
    (length r), L (m x m, unit lower triangular) and E (m x n, echelon).
    """
    U = np.array(A01, dtype=np.uint8) & 1
    m, n = U.shape
    Lc = np.zeros((m, m), dtype=np.uint8)      # coefficients below the diagonal
    upto = [0] * m                             # pivots each row has seen
    P = list(range(m))
    Q: list[int] = []
    r = 0

    def catch_up(i: int) -> None:
        for l in range(upto[i], r):
            if U[i, Q[l]]:
                U[i, :] ^= U[l, :]
                Lc[i, l] = 1
        upto[i] = r

    for j in range(n):
        if r >= m:
            break
        found = -1
        for i in range(r, m):
            catch_up(i)
            if U[i, j]:
                found = i
                break
        if found < 0:
            continue
        P[r] = found
        Q.append(j)
        if found != r:
            U[[r, found], :] = U[[found, r], :]
            Lc[[r, found], :] = Lc[[found, r], :]
            upto[r], upto[found] = upto[found], upto[r]
        r += 1
    for i in range(r, m):
        catch_up(i)
    E = U.copy()
    E[r:, :] = 0
    L = Lc.copy()
    L[:, r:] = 0
    np.fill_diagonal(L, 1)
    return r, np.array(P, dtype=np.int64), np.array(Q, dtype=np.int64), L, E


def compact(L: np.ndarray, E: np.ndarray, r: int) -> np.ndarray:
    """The space-sharing form L\\E: l_ij below the diagonal (columns < r), e_ij elsewhere."""
    m, n = E.shape
    out = E.copy()
    for i in range(m):
        for j in range(min(i, r, n)):
            out[i, j] = L[i, j]
    return out


def perm_from_swaps(P) -> np.ndarray:
    """Permutation matrix of the swap vector: swaps i <-> P[i] applied to I in order."""
    m = len(P)
    order = list(range(m))
    for i, p in enumerate(P):
        order[i], order[p] = order[p], order[i]
    M = np.zeros((m, m), dtype=np.uint8)
    for i, src in enumerate(order):
        M[i, src] = 1
    # order[i] = row of A that ends up at position i, i.e. (P^T A)[i] = A[order[i]];
    # M above is P^T, so P = M^T.
    return M.T.copy()
