"""Pins of the CPU oracle against things other than itself.

Each test ties the oracle to the paper (worked examples under tests/golden),
to brute force over the definitions of Section 2, to a library routine
(numpy integer matmul) or to an independent implementation (oracle/twin.py),
chosen so that a plausible slip -- a dropped L bit, rotation instead of swap,
the wrong bit order, a transposed product, a wrong back-substitution index --
fails at least one of them.  No GPU is needed.
"""
import os

import numpy as np
import pytest

import gf2inputs as gi
import oracle
from oracle import twin
from tests import bruteforce as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    sections, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].rstrip()
            if not line:
                continue
            head = line.split()
            if head[0].isalpha() and not set(head[0]) <= {"0", "1"}:
                cur = head[0]
                sections[cur] = [head[1:]] if len(head) > 1 else []
                continue
            sections[cur].append(head)
    return sections


def _bits(rowstr):
    return [int(c) for c in rowstr]


def _oracle_ple01(U):
    """Run the packed oracle on a 0/1 matrix; return r, P, Q, L, E, compact."""
    U = np.asarray(U, dtype=np.uint8)
    m, n = U.shape
    A = gi.pack(U)
    r, P, Q = oracle.ple(A, m, n, threads=1)
    C = gi.unpack(A, m, n)
    L = np.zeros((m, m), dtype=np.uint8)
    E = np.zeros((m, n), dtype=np.uint8)
    for i in range(m):
        for j in range(n):
            if j < i and j < r:
                L[i, j] = C[i, j]
            elif j >= i:
                E[i, j] = C[i, j]
    np.fill_diagonal(L, 1)
    return r, P, Q[:r], L, E, C


# ---------------------------------------------------------------- bit layout

def test_pack_layout_lsb_first():
    U = np.zeros((2, 130), dtype=np.uint8)
    U[0, 0] = 1
    U[0, 63] = 1
    U[1, 64] = 1
    U[1, 129] = 1
    A = gi.pack(U)
    assert A.shape == (2, 3)
    assert int(A[0, 0]) == (1 | (1 << 63)) and int(A[0, 1]) == 0
    assert int(A[1, 1]) == 1 and int(A[1, 2]) == 2
    assert np.array_equal(gi.unpack(A, 2, 130), U)


def test_generator_deterministic_and_padded():
    a = gi.bernoulli_matrix(37, 100, seed=5)
    b = gi.bernoulli_matrix(37, 100, seed=5)
    assert np.array_equal(a, b)
    assert np.all((a[:, 1] >> np.uint64(36)) == 0)  # columns >= 100 are zero
    # row blocks regenerate independently
    c = gi.bernoulli_matrix(10, 100, seed=5, row0=20)
    assert np.array_equal(a[20:30], c)
    dens = gi.unpack(gi.bernoulli_matrix(256, 256, 7, density_log2=4), 256, 256).mean()
    assert 0.05 < dens < 0.08


# ------------------------------------------------------- the paper's examples

def test_paper_permutation_example():
    """Section 1.2: the 5x5 permutation matrix <-> P = [0, 2, 2, 4, 4].

    Decoding the swap vector must give the printed matrix, and the PLE of
    that matrix (L = E = I) must give back exactly that swap vector."""
    g = _read_golden("paper_permutation_5x5.txt")
    M = np.array([_bits(r[0]) for r in g["matrix"]], dtype=np.uint8)
    swaps = [int(x) for x in g["swaps"][0]]
    assert np.array_equal(twin.perm_from_swaps(swaps), M)
    r, P, Q, L, E, _ = _oracle_ple01(M)
    assert r == 5
    assert P.tolist() == swaps
    assert Q.tolist() == [0, 1, 2, 3, 4]
    assert np.array_equal(L, np.eye(5, dtype=np.uint8))
    assert np.array_equal(E, np.eye(5, dtype=np.uint8))


def test_paper_m4ri_table_figure():
    """Appendix A figure: T[v] = v . A[0:3] with column 0 the most significant
    index bit, and the bold rows are cleared in the first k columns by T[6]."""
    g = _read_golden("paper_m4ri_figure.txt")
    A = np.array([_bits(r[0]) for r in g["A"]], dtype=np.uint8)
    bold = [i for i, r in enumerate(g["A"]) if len(r) > 1 and r[1] == "bold"]
    T = np.array([_bits(r[0]) for r in g["T"]], dtype=np.uint8)
    k, n = 3, A.shape[1]
    top = gi.pack(A[:k])
    for v in range(1 << k):
        coeff = np.array([[(v >> (k - 1 - b)) & 1 for b in range(k)]], dtype=np.uint8)
        prod = oracle.mul(gi.pack(coeff), top, 1, k, n, threads=1)
        assert np.array_equal(gi.unpack(prod, 1, n)[0], T[v]), v
    assert bold == [4, 6]
    for i in bold:
        idx = int("".join(str(b) for b in A[i, :k]), 2)
        assert idx == 6
        cleared = A[i] ^ T[idx]
        assert not cleared[:k].any()
    assert "".join(map(str, A[4] ^ T[6])) == "00000010"


def test_paper_postprocess_example():
    """Section 3.2: with rbar = 3 and the first pivot row starting [1 0 1], a
    later row starting [1 0 1] is cleared by the first pivot row alone, so
    its L bits are [1 0 0]."""
    U = np.array([
        [1, 0, 1, 1, 0, 1],
        [0, 1, 0, 0, 1, 1],
        [0, 0, 1, 1, 1, 0],
        [1, 0, 1, 0, 1, 1],
    ], dtype=np.uint8)
    r, P, Q, L, E, C = _oracle_ple01(U)
    assert Q.tolist()[:3] == [0, 1, 2]
    assert L[3, :3].tolist() == [1, 0, 0]
    assert C[3, :3].tolist() == [1, 0, 0]


def test_swap_not_rotation_hand_example():
    """Rows [010],[001],[100].  Column 0: pivot at row 2, swap 0<->2 gives
    [100],[001],[010] (a rotation would give [100],[010],[001]).  Column 1:
    the first row >= 1 with a 1 is now position 2, so P = [2, 2, 2]."""
    U = np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]], dtype=np.uint8)
    r, P, Q, L, E, _ = _oracle_ple01(U)
    assert r == 3 and P.tolist() == [2, 2, 2] and Q.tolist() == [0, 1, 2]
    assert np.array_equal(E, np.eye(3, dtype=np.uint8))
    assert np.array_equal(L, np.eye(3, dtype=np.uint8))


# ----------------------------------------------------------- brute force pins

SHAPES = [(1, 1), (1, 7), (7, 1), (3, 5), (5, 3), (6, 6), (8, 10), (10, 8), (9, 12), (12, 9)]


@pytest.mark.parametrize("m,n", SHAPES)
@pytest.mark.parametrize("density", [0.5, 0.15])
def test_ple_against_bruteforce(m, n, density):
    rng = np.random.default_rng(1000 * m + n + int(density * 100))
    for trial in range(6):
        U = bf.random01(rng, m, n, density)
        if trial == 1 and m > 2:
            U[m // 2] = 0                               # a zero row
        if trial == 2 and n > 2:
            U[:, n // 2] = 0                            # a zero column
        if trial == 3 and m > 1:
            U[-1] = U[0] ^ U[m // 2]                    # a dependent row
        r, P, Q, L, E, C = _oracle_ple01(U)
        assert r == bf.rank_by_span(U)
        assert Q.tolist() == bf.column_rank_profile(U)
        assert bf.is_echelon(E)
        assert all(E[i, Q[i]] == 1 for i in range(r))
        assert not E[r:].any()
        assert np.array_equal(np.tril(L), L) and all(L[i, i] == 1 for i in range(m))
        assert np.array_equal(L[:, r:], np.eye(m, dtype=np.uint8)[:, r:])  # identity past rank
        Pm = twin.perm_from_swaps(P)
        assert np.array_equal(bf.matmul2(Pm, bf.matmul2(L, E)), U)   # A = P L E


def test_ple_exhaustive_3x3():
    """Every 3x3 matrix: factorisation, rank and profile."""
    for U in bf.all_matrices(3, 3):
        r, P, Q, L, E, C = _oracle_ple01(U)
        assert r == bf.rank_by_span(U)
        assert Q.tolist() == bf.column_rank_profile(U)
        assert np.array_equal(bf.matmul2(twin.perm_from_swaps(P), bf.matmul2(L, E)), U)


@pytest.mark.parametrize("m,n", [(1, 1), (4, 9), (9, 4), (17, 17), (33, 70), (70, 33), (64, 64),
                                 (65, 129), (100, 100)])
@pytest.mark.parametrize("density", [0.5, 0.1, 0.02])
def test_oracle_matches_lazy_twin(m, n, density):
    """Eager packed oracle == lazy unpacked twin (P, Q, rank, L, E)."""
    rng = np.random.default_rng(7 * m + n)
    U = bf.random01(rng, m, n, density)
    if m > 3:
        U[1] = 0
        U[m - 1] = U[0] ^ U[2]
    r, P, Q, L, E, _ = _oracle_ple01(U)
    r2, P2, Q2, L2, E2 = twin.ple(U)
    assert r == r2
    assert P.tolist() == P2.tolist()
    assert Q.tolist() == Q2.tolist()
    assert np.array_equal(E, E2)
    assert np.array_equal(L, L2)


def test_oracle_thread_count_invariant():
    A = gi.bernoulli_matrix(300, 260, seed=3)
    A1, A8 = A.copy(), A.copy()
    r1, P1, Q1 = oracle.ple(A1, 300, 260, threads=1)
    r8, P8, Q8 = oracle.ple(A8, 300, 260, threads=8)
    assert r1 == r8 and np.array_equal(P1, P8) and np.array_equal(Q1, Q8)
    assert np.array_equal(A1, A8)


def test_max_pivots_is_a_prefix():
    """A run limited to k pivots is a prefix of the full elimination."""
    A = gi.bernoulli_matrix(200, 200, seed=9)
    full, part = A.copy(), A.copy()
    r, P, Q = oracle.ple(full, 200, 200, threads=2)
    k, Pk, Qk = oracle.ple(part, 200, 200, max_pivots=50, threads=2)
    assert k == 50
    assert np.array_equal(Pk[:50], P[:50]) and np.array_equal(Qk[:50], Q[:50])


# ------------------------------------------------------------------------ RREF

@pytest.mark.parametrize("m,n", [(3, 5), (6, 6), (9, 12), (12, 9), (10, 10)])
def test_rref_against_bruteforce(m, n):
    rng = np.random.default_rng(31 * m + n)
    for trial in range(5):
        U = bf.random01(rng, m, n, 0.5 if trial % 2 == 0 else 0.2)
        A = gi.pack(U)
        r, Q = oracle.rref(A, m, n, threads=1)
        R = gi.unpack(A, m, n)
        prof = bf.column_rank_profile(U)
        assert Q[:r].tolist() == prof
        assert np.array_equal(R, bf.rref_by_span(U, prof))


# --------------------------------------------------------------------- product

@pytest.mark.parametrize("m,k,n", [(1, 1, 1), (5, 70, 3), (33, 64, 65), (64, 130, 127), (10, 0, 10)])
def test_mul_against_numpy(m, k, n):
    rng = np.random.default_rng(m + 17 * k + 131 * n)
    A = bf.random01(rng, m, k)
    B = bf.random01(rng, k, n)
    C = oracle.mul(gi.pack(A, ld=max(gi.words_for(k), 1)), gi.pack(B, ld=max(gi.words_for(n), 1)),
                   m, k, n, threads=1)
    assert np.array_equal(gi.unpack(C, m, n), bf.matmul2(A, B) if k else np.zeros((m, n), np.uint8))
    C0 = gi.pack(bf.random01(rng, m, n))
    before = gi.unpack(C0, m, n)
    oracle.mul(gi.pack(A, ld=max(gi.words_for(k), 1)), gi.pack(B, ld=max(gi.words_for(n), 1)),
               m, k, n, C=C0, accumulate=True, threads=1)
    want = before ^ (bf.matmul2(A, B) if k else 0)
    assert np.array_equal(gi.unpack(C0, m, n), want)


def test_mul_identity_and_associativity():
    A = gi.bernoulli_matrix(70, 90, 1)
    B = gi.bernoulli_matrix(90, 80, 2)
    C = gi.bernoulli_matrix(80, 50, 3)
    I = gi.pack(np.eye(90, dtype=np.uint8))
    assert np.array_equal(oracle.mul(A, I, 70, 90, 90), A)
    AB_C = oracle.mul(oracle.mul(A, B, 70, 90, 80), C, 70, 80, 50)
    A_BC = oracle.mul(A, oracle.mul(B, C, 90, 80, 50), 70, 90, 50)
    assert np.array_equal(AB_C, A_BC)


# ----------------------------------------------------------------------- solve

@pytest.mark.parametrize("n,nrhs", [(1, 1), (5, 3), (8, 8), (12, 2), (40, 64), (70, 65)])
def test_solve_pins(n, nrhs):
    rng = np.random.default_rng(5 * n + nrhs)
    for trial in range(6):
        U = bf.random01(rng, n, n)
        if trial >= 2 and n > 1:
            U[-1] = U[0]                                  # singular
        Xtrue = bf.random01(rng, n, nrhs)
        Bm = bf.matmul2(U, Xtrue) if trial % 3 != 2 else bf.random01(rng, n, nrhs)
        A = gi.pack(U)
        B = gi.pack(Bm)
        st, r = oracle.solve(A, B, n, nrhs, threads=1)
        if n <= 12:
            assert r == bf.rank_by_span(U)
            consistent = bf.rank_by_span(np.hstack([U, Bm])) == r
        else:
            consistent = None
        if st == oracle.SOLVE_INCONSISTENT:
            assert consistent in (False, None)
            assert consistent is False or trial % 3 == 2
            continue
        X = gi.unpack(B, n, nrhs)
        assert np.array_equal(bf.matmul2(U, X), Bm)
        assert st == (oracle.SOLVE_OK if r == n else oracle.SOLVE_UNDERDETERMINED)
        if consistent is not None:
            assert consistent
        if r == n:
            assert np.array_equal(X, Xtrue)


# ----------------------------------------------- property checkers, with slips

def test_property_checks_accept_oracle_and_reject_slips():
    m, n = 150, 140
    A0 = gi.bernoulli_matrix(m, n, seed=77)
    A0[5] = 0
    LE = A0.copy()
    r, P, Q = oracle.ple(LE, m, n)
    assert oracle.check_ple_all(A0, LE, m, n, P, Q, r) == {
        "structure": 0, "pivot_rule": 0, "freivalds": 0}
    # a dropped L bit
    bad = LE.copy()
    i = m - 1
    bad[i, 0] ^= np.uint64(1 << 3)
    assert oracle.check_freivalds_ple(A0, bad, m, n, P, r) != 0
    # a wrong swap entry (rotation-like slip)
    Pb = P.copy()
    j = int(np.flatnonzero(P[:r] != np.arange(r))[0])
    Pb[j] = j
    assert (oracle.check_freivalds_ple(A0, LE, m, n, Pb, r) != 0
            or oracle.check_pivot_rule(LE, m, Pb, r) != 0)
    # an E entry inside the echelon gap
    bad = LE.copy()
    bad[r - 1, n // 64] ^= np.uint64(1 << (n % 64 - 1))
    assert (oracle.check_ple_structure(bad, m, n, P, Q, r) != 0
            or oracle.check_freivalds_ple(A0, bad, m, n, P, r) != 0)
    # RREF checker
    R = A0.copy()
    rr, QR = oracle.rref(R, m, n)
    assert rr == r and np.array_equal(QR, Q)
    assert oracle.check_rref(R, LE, m, n, Q, r) == 0
    bad = R.copy()
    bad[0, 1] ^= np.uint64(1 << 7)
    assert oracle.check_rref(bad, LE, m, n, Q, r) != 0


def test_pivot_rule_check_catches_a_later_valid_row():
    """A factorisation that is valid (A = P L E) but took a later row as pivot
    must fail the pivot-rule check.  Rows [1 1],[1 0]: the rule takes row 0;
    taking row 1 instead (P = [1, 1]) is another valid PLE."""
    U = np.array([[1, 1], [1, 0]], dtype=np.uint8)
    A0 = gi.pack(U)
    # Valid alternative: swap 0<->1 -> [1 0],[1 1]; E = [[1 0],[0 1]], L = [[1,0],[1,1]]
    alt = gi.pack(np.array([[1, 0], [1, 1]], dtype=np.uint8))
    P = np.array([1, 1], dtype=np.int64)
    Q = np.array([0, 1], dtype=np.int64)
    assert oracle.check_ple_structure(alt, 2, 2, P, Q, 2) == 0
    assert oracle.check_freivalds_ple(A0, alt, 2, 2, P, 2) == 0
    assert oracle.check_pivot_rule(alt, 2, P, 2) != 0
    LE = A0.copy()
    r, P0, Q0 = oracle.ple(LE, 2, 2)
    assert P0.tolist() == [0, 1] and oracle.check_pivot_rule(LE, 2, P0, r) == 0


def test_batch_and_solve_recipes_shape():
    specs = gi.batch_recipe(count=64)
    assert all(64 <= s["m"] <= 1024 and 64 <= s["n"] <= 1024 for s in specs)
    deficient = [s for s in specs if s["zero_rows"]]
    assert 0 < len(deficient) < 64
    assert all(len(s["zero_rows"]) == s["m"] // 10 for s in deficient)
    jobs = gi.solve_stream_recipe(50, rate=1000.0)
    assert all(128 <= j["n"] <= 16384 and 1 <= j["nrhs"] <= 64 for j in jobs)
    assert all(jobs[i]["t"] < jobs[i + 1]["t"] for i in range(49))


def test_row_weight_generator_exact_weights():
    """The sparse workload of Section 4's Figure: exactly w ones per row,
    distinct columns, padding clear, deterministic per seed."""
    for m, n, w in [(50, 70, 0), (50, 70, 1), (40, 130, 17), (30, 64, 64), (200, 1000, 40)]:
        A = gi.row_weight_matrix(m, n, w, seed=9)
        U = gi.unpack(A, m, n)
        assert (U.sum(axis=1) == w).all()
        assert np.array_equal(A, gi.row_weight_matrix(m, n, w, seed=9))
        if n % 64:
            assert not (A[:, -1] & np.uint64(~gi.pad_mask(n) & 0xFFFFFFFFFFFFFFFF)).any()
    # columns are spread: every column of a 2000 x 100 draw with w = 50 is hit
    U = gi.unpack(gi.row_weight_matrix(2000, 100, 50, seed=3), 2000, 100)
    assert (U.sum(axis=0) > 700).all() and (U.sum(axis=0) < 1300).all()
