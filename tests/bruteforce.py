"""Brute-force references for tiny GF(2) matrices (pure Python/numpy).

These enumerate row spaces and column subsets directly from the definitions
of Section 2 (column rank profile, row echelon form, reduced row echelon
form, PLE decomposition) and are used only to pin the oracle.
"""
from __future__ import annotations

import itertools

import numpy as np


def rows_as_ints(U: np.ndarray) -> list[int]:
    """Rows of a 0/1 matrix as Python ints (bit j = column j)."""
    out = []
    for row in np.asarray(U, dtype=np.uint8):
        v = 0
        for j, b in enumerate(row):
            if b:
                v |= 1 << j
        out.append(v)
    return out


def span(vectors: list[int]) -> set[int]:
    """All XOR combinations of the given vectors (2^k of them for k vectors)."""
    s = {0}
    for v in vectors:
        s |= {x ^ v for x in s}
    return s


def rank_by_span(U: np.ndarray) -> int:
    """Rank = log2 of the size of the row space (enumerated)."""
    size = len(span(rows_as_ints(U)))
    r = size.bit_length() - 1
    assert 1 << r == size
    return r


def column_rank_profile(U: np.ndarray) -> list[int]:
    """Lexicographically smallest set of independent columns (Definition
    "Column rank profile"): greedily keep column j when it raises the rank of
    the columns kept so far; the rank is computed by span enumeration."""
    U = np.asarray(U, dtype=np.uint8)
    kept: list[int] = []
    r = 0
    for j in range(U.shape[1]):
        trial = kept + [j]
        rr = rank_by_span(U[:, trial].T)
        if rr > r:
            kept, r = trial, rr
    return kept


def rref_by_span(U: np.ndarray, pivots: list[int]) -> np.ndarray:
    """The RREF, found as the unique row-space vectors whose restriction to
    the pivot columns is a unit vector (Definition "Reduced Row Echelon Form"
    and its uniqueness)."""
    U = np.asarray(U, dtype=np.uint8)
    m, n = U.shape
    sp = span(rows_as_ints(U))
    out = np.zeros((m, n), dtype=np.uint8)
    for p, qp in enumerate(pivots):
        want = 1 << qp
        mask = sum(1 << q for q in pivots)
        cands = [v for v in sp if (v & mask) == want and (v & ((1 << qp) - 1)) == 0]
        assert len(cands) == 1, cands
        v = cands[0]
        out[p] = [(v >> j) & 1 for j in range(n)]
    return out


def is_echelon(E: np.ndarray) -> bool:
    """Definition "Row Echelon Form": zero rows at the bottom, leading entries
    strictly moving right."""
    last = -1
    seen_zero = False
    for row in np.asarray(E, dtype=np.uint8):
        nz = np.flatnonzero(row)
        if len(nz) == 0:
            seen_zero = True
            continue
        if seen_zero or nz[0] <= last:
            return False
        last = nz[0]
    return True


def matmul2(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Product over GF(2) through numpy's integer matmul, reduced mod 2."""
    return (np.asarray(A, dtype=np.int64) @ np.asarray(B, dtype=np.int64) % 2).astype(np.uint8)


def random01(rng: np.random.Generator, m: int, n: int, density: float = 0.5) -> np.ndarray:
    return (rng.random((m, n)) < density).astype(np.uint8)


def all_matrices(m: int, n: int):
    """Every m x n 0/1 matrix (for exhaustive checks on very small shapes)."""
    for bits in itertools.product((0, 1), repeat=m * n):
        yield np.array(bits, dtype=np.uint8).reshape(m, n)
