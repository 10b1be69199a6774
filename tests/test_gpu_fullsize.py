"""Full-size parity: the workloads the benchmark times, in the same launch path.

At 32768^2 and 65536^2 the eager oracle would take minutes, so every output
is checked through properties that pin it uniquely (oracle/gf2_checks.c:
echelon structure, Freivalds' A = P L E with 64 random vectors, the pivot
rule through the L bits, and U R = E for the RREF), plus an exact comparison
with the oracle run on the leading 1024 columns: the elimination of those
columns depends on nothing to their right, so P, Q, the first pivots' rows
of E and the first L columns must match bit for bit.
"""
import numpy as np
import pytest

import gf2inputs as gi
import oracle
from tests.gpu_util import to_dev, to_host, vec_dev

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def h():
    import paper_1111_6549_gb300 as g
    return g.Handle()


def prefix_check(A, LE, P, Q, r, m, n, c0=1024):
    Ap = np.ascontiguousarray(A[:, : c0 // 64])
    r0, P0, Q0 = oracle.ple(Ap, m, c0)
    assert np.array_equal(P[:r0], P0[:r0])
    assert np.array_equal(Q[:r0], Q0[:r0])
    if r0 < r:
        assert Q[r0] >= c0
    for p in range(r0, r):                       # later swaps move the prefix's rows too
        q = int(P[p])
        if q != p:
            Ap[[p, q]] = Ap[[q, p]]
    assert np.array_equal(LE[:r0, : c0 // 64], Ap[:r0])
    wr = r0 // 64
    assert np.array_equal(LE[r0:, :wr], Ap[r0:, :wr])
    if r0 % 64:
        mask = np.uint64((1 << (r0 % 64)) - 1)
        assert np.array_equal(LE[r0:, wr] & mask, Ap[r0:, wr] & mask)


def ple_and_rref_checked(h, A, m, n, expect_rank=None, block=None):
    if block is not None:
        import paper_1111_6549_gb300 as g
        h = g.Handle()
        h.set_option(g.OPT_PLE_BLOCK, block)
    dA = to_dev(A)
    P, Q = vec_dev(m), vec_dev(min(m, n))
    r = h.ple(dA, m, n, P, Q)
    LE = to_host(dA, gi.words_for(n))
    del dA
    Ph, Qh = P.cpu().numpy()[:m], Q.cpu().numpy()[: min(m, n)]
    if expect_rank is not None:
        assert r == expect_rank
    assert oracle.check_ple_all(A, LE, m, n, Ph, Qh, r) == {
        "structure": 0, "pivot_rule": 0, "freivalds": 0}
    prefix_check(A, LE, Ph, Qh, r, m, n)
    dR = to_dev(A)
    Q2 = vec_dev(min(m, n))
    r2 = h.rref(dR, m, n, Q2)
    R = to_host(dR, gi.words_for(n))
    del dR
    assert r2 == r
    assert np.array_equal(Q2.cpu().numpy()[: min(m, n)], Qh)
    assert oracle.check_rref(R, LE, m, n, Qh, r) == 0
    # M4RI (Algorithm 8) reaches the same unique RREF
    dM = to_dev(A)
    Q3 = vec_dev(min(m, n))
    r3 = h.rref_m4ri(dM, m, n, Q3)
    M = to_host(dM, gi.words_for(n))
    del dM
    assert r3 == r and np.array_equal(Q3.cpu().numpy()[: min(m, n)], Qh)
    assert oracle.check_rref(M, LE, m, n, Qh, r) == 0
    return r


@pytest.mark.parametrize("n", [32768, 65536])
def test_dense_square_fullsize(h, n):
    A = gi.dense_square(n)
    r = ple_and_rref_checked(h, A, n, n)
    assert n - 8 <= r <= n          # a random square GF(2) matrix is nearly full rank


def test_structured_rank_8192(h):
    X, Y = gi.structured_factors()
    A = oracle.mul(X, Y, 16384, 8192, 32768)
    ple_and_rref_checked(h, A, 16384, 32768, expect_rank=8192)


def test_sparse_square_32768(h):
    A = gi.sparse_square(32768)
    ple_and_rref_checked(h, A, 32768, 32768)


@pytest.mark.parametrize("block", [8192, 16384])
def test_dense_square_blocked_fullsize(h, block):
    """The blocked PLE (block trailing updates through the library GEMM) at 65536^2."""
    A = gi.dense_square(65536)
    r = ple_and_rref_checked(h, A, 65536, 65536, block=block)
    assert 65536 - 8 <= r <= 65536
