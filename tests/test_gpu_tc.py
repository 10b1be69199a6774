"""The alternative forms of the product and of the trailing updates -- the
tensor-core (tcgen05) kernels, the library GEMM, the TMA-staged and the
paired 64-byte-tile table updates: bit-exact against the oracle, like the
default forms."""
import numpy as np
import pytest

import gf2inputs as gi
import oracle
from tests.gpu_util import to_dev, to_host, vec_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    import paper_1111_6549_gb300 as g
    hh = g.Handle()
    hh.set_option(g.OPT_TC_MUL, 1)
    return hh


@pytest.mark.parametrize("m,k,n", [(128, 64, 256), (1, 1, 1), (300, 70, 300), (129, 65, 257),
                                   (1000, 1000, 1000), (513, 2049, 300), (64, 0, 64), (2048, 130, 4100)])
@pytest.mark.parametrize("accumulate", [False, True])
def test_tc_mul(h, m, k, n, accumulate):
    A = gi.bernoulli_matrix(m, k, 11) if k else np.zeros((m, 1), np.uint64)
    B = gi.bernoulli_matrix(k, n, 12) if k else np.zeros((1, gi.words_for(n)), np.uint64)
    C0 = gi.bernoulli_matrix(m, n, 13)
    dC = to_dev(C0)
    h.mul(dC, to_dev(A), to_dev(B), m, k, n, accumulate=accumulate)
    want = C0.copy() if accumulate else np.zeros_like(C0)
    if k:
        oracle.mul(A, B, m, k, n, C=want, accumulate=accumulate)
    assert np.array_equal(to_host(dC), want)


@pytest.mark.parametrize("kind,m,n", [("dense", 300, 300), ("dense", 1000, 1500), ("lowrank", 700, 900),
                                      ("dense", 2048, 2048)])
def test_tc_update_ple_and_rref(kind, m, n):
    import paper_1111_6549_gb300 as g
    hh = g.Handle()
    hh.set_option(g.OPT_TC_UPDATE, 1)
    if kind == "dense":
        A = gi.bernoulli_matrix(m, n, m + n)
    else:
        k = min(m, n) // 3
        A = oracle.mul(gi.bernoulli_matrix(m, k, 1), gi.bernoulli_matrix(k, n, 2), m, k, n)
    dA = to_dev(A)
    P, Q = vec_dev(m), vec_dev(min(m, n))
    r = hh.ple(dA, m, n, P, Q)
    LE = A.copy()
    r0, P0, Q0 = oracle.ple(LE, m, n)
    assert r == r0
    assert np.array_equal(P.cpu().numpy()[:m], P0) and np.array_equal(Q.cpu().numpy()[:min(m, n)], Q0)
    assert np.array_equal(to_host(dA, gi.words_for(n)), LE)
    dR = to_dev(A)
    r2 = hh.rref(dR, m, n, Q)
    R0 = A.copy()
    oracle.rref(R0, m, n)
    assert r2 == r0 and np.array_equal(to_host(dR, gi.words_for(n)), R0)


@pytest.mark.parametrize("m,n", [(300, 1100), (1000, 1500), (2048, 2048), (4099, 1030)])
def test_tma_update_ple_rref_and_mul(m, n):
    """The TMA-staged form of the table update (GF2_OPT_TMA_UPDATE)."""
    import paper_1111_6549_gb300 as g
    hh = g.Handle()
    hh.set_option(g.OPT_TMA_UPDATE, 1)
    A = gi.bernoulli_matrix(m, n, 7 * m + n)
    dA = to_dev(A)
    P, Q = vec_dev(m), vec_dev(min(m, n))
    r = hh.ple(dA, m, n, P, Q)
    LE = A.copy()
    r0, P0, Q0 = oracle.ple(LE, m, n)
    assert r == r0 and np.array_equal(P.cpu().numpy()[:m], P0)
    assert np.array_equal(to_host(dA, gi.words_for(n)), LE)
    dR = to_dev(A)
    assert hh.rref(dR, m, n, Q) == r0
    R0 = A.copy()
    oracle.rref(R0, m, n)
    assert np.array_equal(to_host(dR, gi.words_for(n)), R0)
    k = 200
    B = gi.bernoulli_matrix(k, n, 3)
    X = gi.bernoulli_matrix(m, k, 4)
    C0 = gi.bernoulli_matrix(m, n, 5)
    dC = to_dev(C0)
    hh.mul(dC, to_dev(X), to_dev(B), m, k, n, accumulate=True)
    want = C0.copy()
    oracle.mul(X, B, m, k, n, C=want, accumulate=True)
    assert np.array_equal(to_host(dC), want)


@pytest.mark.parametrize("m,n", [(300, 1100), (1000, 1500), (2048, 2048), (4099, 1030), (2500, 3000)])
def test_paired_update_ple_rref_m4ri_and_mul(m, n):
    """The paired 64-byte-tile form of the table update (GF2_OPT_WIDE_UPDATE = 0;
    the default runs 128-byte tiles with nine tables)."""
    import paper_1111_6549_gb300 as g
    hh = g.Handle()
    hh.set_option(g.OPT_WIDE_UPDATE, 0)
    A = gi.bernoulli_matrix(m, n, 5 * m + n)
    dA = to_dev(A)
    P, Q = vec_dev(m), vec_dev(min(m, n))
    r = hh.ple(dA, m, n, P, Q)
    LE = A.copy()
    r0, P0, Q0 = oracle.ple(LE, m, n)
    assert r == r0 and np.array_equal(P.cpu().numpy()[:m], P0)
    assert np.array_equal(to_host(dA, gi.words_for(n)), LE)
    R0 = A.copy()
    oracle.rref(R0, m, n)
    dR = to_dev(A)
    assert hh.rref(dR, m, n, Q) == r0
    assert np.array_equal(to_host(dR, gi.words_for(n)), R0)
    dM = to_dev(A)
    assert hh.rref_m4ri(dM, m, n, Q) == r0
    assert np.array_equal(to_host(dM, gi.words_for(n)), R0)
    k = 200
    B = gi.bernoulli_matrix(k, n, 3)
    X = gi.bernoulli_matrix(m, k, 4)
    C0 = gi.bernoulli_matrix(m, n, 5)
    dC = to_dev(C0)
    hh.mul(dC, to_dev(X), to_dev(B), m, k, n, accumulate=True)
    want = C0.copy()
    oracle.mul(X, B, m, k, n, C=want, accumulate=True)
    assert np.array_equal(to_host(dC), want)


@pytest.mark.parametrize("m,k,n", [(1, 1, 1), (128, 64, 256), (300, 70, 300), (129, 65, 257), (1000, 5000, 1000),
                                   (513, 4099, 300), (2048, 130, 4100), (64, 0, 64)])
@pytest.mark.parametrize("accumulate", [False, True])
@pytest.mark.parametrize("fmt", [8, 4])
def test_mul_through_library_gemm(m, k, n, accumulate, fmt):
    """gf2_mul through the exact library GEMM (forced for every k), with FP8
    E4M3 operands and with block-scaled FP4 E2M1 operands (only when the
    library GEMM is built in)."""
    import paper_1111_6549_gb300 as g
    from tests.gpu_util import library_gemm_available
    if not library_gemm_available():
        pytest.skip("library GEMM not built in (GF2_WITH_CUBLASLT)")
    hh = g.Handle()
    hh.set_option(g.OPT_MUL_GEMM_MIN_K, 1)
    hh.set_option(g.OPT_MUL_GEMM_FORMAT, fmt)
    A = gi.bernoulli_matrix(m, k, 21) if k else np.zeros((m, 1), np.uint64)
    B = gi.bernoulli_matrix(k, n, 22) if k else np.zeros((1, gi.words_for(n)), np.uint64)
    C0 = gi.bernoulli_matrix(m, n, 23)
    dC = to_dev(C0)
    hh.mul(dC, to_dev(A), to_dev(B), m, k, n, accumulate=accumulate)
    want = C0.copy() if accumulate else np.zeros_like(C0)
    if k:
        oracle.mul(A, B, m, k, n, C=want, accumulate=accumulate)
    assert np.array_equal(to_host(dC), want)


def test_mul_default_large_k_matches_oracle():
    """Default options: a large inner dimension takes the own tcgen05 FP4 GEMM."""
    import paper_1111_6549_gb300 as g
    hh = g.Handle()
    m, k, n = 700, 9000, 1100
    A, B = gi.bernoulli_matrix(m, k, 31), gi.bernoulli_matrix(k, n, 32)
    dC = to_dev(np.zeros((m, gi.words_for(n)), np.uint64))
    hh.mul(dC, to_dev(A), to_dev(B), m, k, n)
    assert np.array_equal(to_host(dC), oracle.mul(A, B, m, k, n))


@pytest.mark.parametrize("m,n", [(300, 1100), (1000, 1500), (2048, 2048)])
def test_naive_update_ple_and_rref(m, n):
    """The plain baseline (GF2_OPT_NAIVE_UPDATE: generator rows added one by
    one, no tables) gives the same unique PLE and RREF."""
    import paper_1111_6549_gb300 as g
    hh = g.Handle()
    hh.set_option(g.OPT_NAIVE_UPDATE, 1)
    hh.set_option(g.OPT_LOOKAHEAD, 0)
    A = gi.bernoulli_matrix(m, n, 5 * m + n)
    dA = to_dev(A)
    P, Q = vec_dev(m), vec_dev(min(m, n))
    r = hh.ple(dA, m, n, P, Q)
    LE = A.copy()
    r0, P0, Q0 = oracle.ple(LE, m, n)
    assert r == r0 and np.array_equal(P.cpu().numpy()[:m], P0)
    assert np.array_equal(to_host(dA, gi.words_for(n)), LE)
    dR = to_dev(A)
    assert hh.rref(dR, m, n, Q) == r0
    R0 = A.copy()
    oracle.rref(R0, m, n)
    assert np.array_equal(to_host(dR, gi.words_for(n)), R0)


@pytest.mark.parametrize("m,n,block", [(1000, 1500, 0), (2048, 2048, 512), (3000, 2500, 1024), (700, 900, 128)])
def test_pdl_launches_ple_rref_mul(m, n, block):
    """GF2_OPT_PDL: every kernel scheduled while its predecessor on the stream
    runs and waiting on the device for it -- the same unique results, with the
    blocked PLE and RREF (TRSM leaves and products) and the look-ahead."""
    import paper_1111_6549_gb300 as g
    hh = g.Handle()
    hh.set_option(g.OPT_PDL, 1)
    if block:
        hh.set_option(g.OPT_PLE_BLOCK, block)
        hh.set_option(g.OPT_RREF_BLOCK, block)
        hh.set_option(g.OPT_MUL_GEMM_MIN_K, 256)
    A = gi.bernoulli_matrix(m, n, 9 * m + n)
    dA = to_dev(A)
    P, Q = vec_dev(m), vec_dev(min(m, n))
    r = hh.ple(dA, m, n, P, Q)
    LE = A.copy()
    r0, P0, Q0 = oracle.ple(LE, m, n)
    assert r == r0 and np.array_equal(P.cpu().numpy()[:m], P0)
    assert np.array_equal(Q.cpu().numpy()[:min(m, n)], Q0)
    assert np.array_equal(to_host(dA, gi.words_for(n)), LE)
    dR = to_dev(A)
    assert hh.rref(dR, m, n, Q) == r0
    R0 = A.copy()
    oracle.rref(R0, m, n)
    assert np.array_equal(to_host(dR, gi.words_for(n)), R0)
    B = gi.bernoulli_matrix(n, 300, 3)
    dC = to_dev(np.zeros((m, gi.words_for(300)), np.uint64))
    hh.mul(dC, to_dev(A), to_dev(B), m, n, 300)
    assert np.array_equal(to_host(dC), oracle.mul(A, B, m, n, 300))


def test_profiling_timeline():
    """Profiling level 4 keeps one (kind, start, end) record per launch."""
    import paper_1111_6549_gb300 as g
    hh = g.Handle()
    m = n = 1024
    A = gi.bernoulli_matrix(m, n, 77)
    dA = to_dev(A)
    P, Q = vec_dev(m), vec_dev(n)
    hh.reset_stats()
    hh.set_profiling(4)
    hh.ple(dA, m, n, P, Q)
    tl = hh.timeline()
    st = hh.stats()
    assert 0 < len(tl) <= st["kernel_launches"]
    kinds = {k for k, _, _ in tl}
    assert {0, 1, 2} <= kinds
    assert all(0.0 <= t0 <= t1 for _, t0, t1 in tl)
