"""The blocked PLE (GF2_OPT_PLE_BLOCK): stripes decomposed block by block,
each block's trailing update applied at once (TRSM + GF(2) product).  The
decomposition is unique, so every output must equal the oracle's bit for bit,
for every block width, including rank-deficient blocks whose pivot rows are
not word aligned."""
import numpy as np
import pytest

import gf2inputs as gi
import oracle
from tests.gpu_util import to_dev, to_host, vec_dev
from tests.gpu_util import library_gemm_available
from tests.test_gpu_parity import assert_ple_equal, make, ref_ple

pytestmark = pytest.mark.gpu


def handle(block, gemm_min_k=None, fmt=0, rref_block=None):
    import paper_1111_6549_gb300 as g
    h = g.Handle()
    h.set_option(g.OPT_PLE_BLOCK, block)
    h.set_option(g.OPT_RREF_BLOCK, block if rref_block is None else rref_block)
    h.set_option(g.OPT_MUL_GEMM_FORMAT, fmt)
    if gemm_min_k is not None:
        h.set_option(g.OPT_MUL_GEMM_MIN_K, gemm_min_k)
    return h


def run(h, A, m, n, ld_extra=0):
    W = gi.words_for(n)
    dA = to_dev(A, W + ld_extra)
    P, Q = vec_dev(m), vec_dev(min(m, n))
    r = h.ple(dA, m, n, P, Q)
    return r, to_host(dA, W), P.cpu().numpy()[:m], Q.cpu().numpy()[:min(m, n)]


@pytest.mark.parametrize("block", [64, 128, 256, 1024])
@pytest.mark.parametrize("kind,m,n", [("dense", 1000, 1500), ("lowrank", 700, 900), ("lastrow_pivot", 600, 800),
                                      ("sparse", 900, 1300), ("zerocols", 800, 1000), ("dense", 1500, 700),
                                      ("duprows", 640, 640)])
def test_blocked_ple_matches_oracle(block, kind, m, n):
    A = make(kind, m, n, seed=block + m)
    assert_ple_equal(run(handle(block), A, m, n), ref_ple(A, m, n))


@pytest.mark.parametrize("gemm_min_k,fmt", [(1, 0), (1, 8), (1, 4), (0, 0)])
def test_blocked_ple_gemm_and_table_products(gemm_min_k, fmt):
    if fmt and not library_gemm_available():
        pytest.skip("library GEMM not built in (GF2_WITH_CUBLASLT)")
    """The block's product through the FP8 or FP4 GEMM (min k 1) and through the tables (0)."""
    m, n = 3000, 2049
    A = make("dense", m, n, seed=3)
    assert_ple_equal(run(handle(512, gemm_min_k, fmt), A, m, n, ld_extra=1), ref_ple(A, m, n))


def test_blocked_rref_and_solve():
    h = handle(256, 1)
    m, n = 2000, 2300
    A = make("lowrank", m, n, seed=9)
    dR = to_dev(A)
    Q = vec_dev(min(m, n))
    r = h.rref(dR, m, n, Q)
    R0 = A.copy()
    r0, Q0 = oracle.rref(R0, m, n)
    assert r == r0 and np.array_equal(to_host(dR, gi.words_for(n)), R0)
    nn, nrhs = 1500, 40
    As = make("dense", nn, nn, seed=4)
    Bs = gi.bernoulli_matrix(nn, nrhs, 5)
    dA, dB = to_dev(As), to_dev(Bs)
    st = h.solve(dA, dB, nn, nrhs)
    A0, B0 = As.copy(), Bs.copy()
    st0, _ = oracle.solve(A0, B0, nn, nrhs)
    assert st == st0
    if st0 != oracle.SOLVE_INCONSISTENT:
        assert np.array_equal(to_host(dB, gi.words_for(nrhs)), B0)


@pytest.mark.parametrize("rref_block", [128, 64])
@pytest.mark.parametrize("m,n", [(700, 1500), (1500, 700), (640, 640)])
def test_blocked_rref_wide_tall_and_exhausted(m, n, rref_block):
    """Rank reaching m before the last block (wide), tall, and square: the RREF
    built on the blocked PLE's stripe records, recursive down to one or two
    stripes per block."""
    h = handle(128, 1, rref_block=rref_block)
    A = make("dense", m, n, seed=m + 3 * n)
    dR = to_dev(A)
    Q = vec_dev(min(m, n))
    r = h.rref(dR, m, n, Q)
    R0 = A.copy()
    r0, Q0 = oracle.rref(R0, m, n)
    assert r == r0 and np.array_equal(Q.cpu().numpy()[:min(m, n)], Q0)
    assert np.array_equal(to_host(dR, gi.words_for(n)), R0)


@pytest.mark.parametrize("rref_block", [640, 128])
@pytest.mark.parametrize("dups", [(), (700,), (640,), (767, 768), (900, 1000, 1270, 1279), (1279,)])
def test_blocked_rref_pivot_gaps(dups, rref_block):
    """The right half's pivot columns with gaps (a column equal to an earlier
    one is no pivot): the gathered bits then come from scattered columns, and
    the left stripes skip only the words before the first gap."""
    m = n = 1280
    A = make("dense", m, n, seed=sum(dups) + 11)
    U = gi.unpack(A, m, n)
    for c in dups:
        U[:, c] = U[:, c - 37]
    A = gi.pack(U, A.shape[1])
    h = handle(640, 1, 0, rref_block)
    dR = to_dev(A)
    Q = vec_dev(n)
    r = h.rref(dR, m, n, Q)
    R0 = A.copy()
    r0, Q0 = oracle.rref(R0, m, n)
    assert r == r0 and np.array_equal(Q.cpu().numpy()[:r0], Q0[:r0])
    assert not set(dups) & set(Q0[:r0].tolist())
    assert np.array_equal(to_host(dR, gi.words_for(n)), R0)


@pytest.mark.parametrize("leaf", [1024, 2048, 4096])
@pytest.mark.parametrize("kind,m,n,block", [("dense", 9000, 9000, 8192), ("lowrank", 9100, 9000, 8192),
                                            ("dense", 8800, 12345, 4096), ("sparse", 5000, 5100, 4352)])
def test_blocked_ple_trsm_leaf_sizes(leaf, kind, m, n, block):
    """The fused TRSM leaves at every size (GF2_OPT_TRSM_LEAF): diagonal blocks
    of 8192 rows halved down to the leaf, blocks of fewer rows than a leaf
    (the low-rank and sparse cases: ragged leaves), and an odd number of
    trailing words (the last leaf CTA owns one word)."""
    import paper_1111_6549_gb300 as g
    h = handle(block)
    h.set_option(g.OPT_TRSM_LEAF, leaf)
    A = make(kind, m, n, seed=leaf + m + n)
    assert_ple_equal(run(h, A, m, n, ld_extra=1), ref_ple(A, m, n))


@pytest.mark.parametrize("compact,leaf", [(1, 1), (0, 1), (0, 0)])
@pytest.mark.parametrize("kind,m,n,rref_block,dups", [
    ("dense", 9000, 9000, 8192, ()), ("lowrank", 9000, 9500, 4096, ()), ("dense", 6000, 13000, 8192, ()),
    ("dense", 13000, 6000, 8192, ()), ("dense", 8200, 8200, 8192, (4000, 8191, 8192)),
    ("sparse", 5000, 7000, 2048, (100, 3000))])
def test_rref_leaf_base_blocks(compact, leaf, kind, m, n, rref_block, dups):
    """The RREF recovery three ways: compact (GF2_OPT_RREF_COMPACT, only the
    non-pivot columns solved, leaves of rref_block rows), and stripe-wise with
    each base block reduced by the fused back-substitution leaf
    (GF2_OPT_RREF_LEAF 1) or by one table pass per stripe (0).  Full blocks of
    8192 pivot rows, rank-deficient and wide matrices (the words past the
    skipped pivot columns reduced by a second leaf launch), tall ones, and
    pivot gaps from repeated columns."""
    import paper_1111_6549_gb300 as g
    A = make(kind, m, n, seed=m + n + rref_block + len(dups))
    if dups:
        U = gi.unpack(A, m, n)
        for c in dups:
            U[:, c] = U[:, c - 37]
        A = gi.pack(U, A.shape[1])
    h = handle(0, rref_block=rref_block)
    h.set_option(g.OPT_RREF_LEAF, leaf)
    h.set_option(g.OPT_RREF_COMPACT, compact)
    dR = to_dev(A, gi.words_for(n) + 1)
    Q = vec_dev(min(m, n))
    r = h.rref(dR, m, n, Q)
    R0 = A.copy()
    r0, Q0 = oracle.rref(R0, m, n)
    assert r == r0 and np.array_equal(Q.cpu().numpy()[:r0], Q0[:r0])
    assert np.array_equal(to_host(dR, gi.words_for(n)), R0)


@pytest.mark.parametrize("leaf_rows", [64, 128, 1024])
@pytest.mark.parametrize("kind,m,n", [("dense", 700, 900), ("lowrank", 900, 700), ("zerorows", 600, 600),
                                      ("dense", 1200, 500), ("dense", 500, 1200), ("sparse", 800, 1000),
                                      ("zero", 300, 400), ("dense", 1, 130), ("dense", 130, 1)])
def test_rref_compact_shapes(leaf_rows, kind, m, n):
    """The compact recovery on small shapes, with leaves of 64 (one step, so
    every reduction goes through the products), 128 and 1024 rows: full
    column rank (no non-pivot column: only the identity is written), the zero
    matrix (rank 0), single rows and columns."""
    import paper_1111_6549_gb300 as g
    A = np.zeros((m, gi.words_for(n)), dtype=np.uint64) if kind == "zero" else make(kind, m, n, seed=m + 3 * n)
    h = handle(0, rref_block=leaf_rows)
    dR = to_dev(A)
    Q = vec_dev(min(m, n))
    r = h.rref(dR, m, n, Q)
    R0 = A.copy()
    r0, Q0 = oracle.rref(R0, m, n)
    assert r == r0 and np.array_equal(Q.cpu().numpy()[:r0], Q0[:r0])
    assert np.array_equal(to_host(dR, gi.words_for(n)), R0)


@pytest.mark.parametrize("m,n,dups,leaf_rows", [(3000, 3000, (100, 2000, 2999), 64), (3000, 3000, (1500,), 1024),
                                                (2600, 2600, tuple(range(300, 2600, 300)), 128),
                                                (2600, 2600, tuple(range(300, 2600, 260)), 128),
                                                (9000, 9000, (8999,), -1), (700, 4000, (), 256)])
def test_rref_compact_narrow_joins(m, n, dups, leaf_rows):
    """Compact recovery with few non-pivot columns (columns repeated from
    earlier ones): the joins take the narrow parity path up to eight such
    columns (the 8-column case) and the GEMM beyond (the 9-column case and the
    wide matrix); leaves of 64 rows make every reduction a join."""
    import paper_1111_6549_gb300 as g
    A = make("dense", m, n, seed=m + n + len(dups))
    if dups:
        U = gi.unpack(A, m, n)
        for c in dups:
            U[:, c] = U[:, c - 37]
        A = gi.pack(U, A.shape[1])
    h = g.Handle()
    h.set_option(g.OPT_RREF_BLOCK, leaf_rows)
    dR = to_dev(A)
    Q = vec_dev(min(m, n))
    r = h.rref(dR, m, n, Q)
    R0 = A.copy()
    r0, Q0 = oracle.rref(R0, m, n)
    assert r == r0 and np.array_equal(Q.cpu().numpy()[:r0], Q0[:r0])
    assert np.array_equal(to_host(dR, gi.words_for(n)), R0)


@pytest.mark.parametrize("bad", [0, 512, 1000, 8192, -1])
def test_trsm_leaf_option_rejects_other_sizes(bad):
    import paper_1111_6549_gb300 as g
    h = g.Handle()
    with pytest.raises(g.GF2Error):
        h.set_option(g.OPT_TRSM_LEAF, bad)


@pytest.mark.parametrize("block", [64, 192, 256])
@pytest.mark.parametrize("kind,m,n", [("dense", 1000, 1500), ("lowrank", 700, 900), ("lastrow_pivot", 600, 800),
                                      ("zerocols", 800, 1000), ("dense", 1500, 700), ("duprows", 640, 640)])
def test_recursive_ple_matches_oracle(block, kind, m, n):
    """Algorithm 3's recursion (GF2_OPT_PLE_RECURSIVE): columns halved down to
    the block width, each left half's trailing update on its sibling only."""
    import paper_1111_6549_gb300 as g
    h = handle(block)
    h.set_option(g.OPT_PLE_RECURSIVE, 1)
    A = make(kind, m, n, seed=block + 7 * m)
    assert_ple_equal(run(h, A, m, n, ld_extra=1), ref_ple(A, m, n))


def test_recursive_ple_rref_and_solve():
    """The RREF and the solve on top of the recursive PLE."""
    import paper_1111_6549_gb300 as g
    h = handle(128, 1)
    h.set_option(g.OPT_PLE_RECURSIVE, 1)
    m, n = 1800, 2100
    A = make("lowrank", m, n, seed=21)
    dR = to_dev(A)
    Q = vec_dev(min(m, n))
    r = h.rref(dR, m, n, Q)
    R0 = A.copy()
    r0, Q0 = oracle.rref(R0, m, n)
    assert r == r0 and np.array_equal(to_host(dR, gi.words_for(n)), R0)
    nn, nrhs = 1300, 33
    As = make("dense", nn, nn, seed=22)
    Bs = gi.bernoulli_matrix(nn, nrhs, 23)
    dA, dB = to_dev(As), to_dev(Bs)
    st = h.solve(dA, dB, nn, nrhs)
    A0, B0 = As.copy(), Bs.copy()
    st0, _ = oracle.solve(A0, B0, nn, nrhs)
    assert st == st0
    if st0 != oracle.SOLVE_INCONSISTENT:
        assert np.array_equal(to_host(dB, gi.words_for(nrhs)), B0)
