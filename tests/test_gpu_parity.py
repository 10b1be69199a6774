"""Bit-exact parity of the CUDA path (through the C ABI) with the CPU oracle.

Sizes here finish in the oracle within seconds and still span many 64-column
stripes, several update tiles and ragged edges; the inputs cover the
degenerate cases of the method (rank-deficient stripes, zero columns that
force the block-wide pivot search, pivots far below the window, empty and
one-row/one-column matrices, odd leading dimensions).
"""
import zlib

import numpy as np
import pytest

import gf2inputs as gi
import oracle
from tests.gpu_util import to_dev, to_host, vec_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    import paper_1111_6549_gb300 as g
    return g.Handle()


def make(kind: str, m: int, n: int, seed: int) -> np.ndarray:
    if kind == "dense":
        return gi.bernoulli_matrix(m, n, seed)
    if kind == "sparse":
        return gi.bernoulli_matrix(m, n, seed, density_log2=4)
    if kind == "lowrank":
        k = max(1, min(m, n) // 3)
        X = gi.bernoulli_matrix(m, k, seed)
        Y = gi.bernoulli_matrix(k, n, seed + 1)
        return oracle.mul(X, Y, m, k, n)
    if kind == "zerorows":
        A = gi.bernoulli_matrix(m, n, seed)
        A[::3] = 0
        return A
    if kind == "duprows":
        A = gi.bernoulli_matrix(m, n, seed)
        A[1::2] = A[0:(m // 2) * 2:2][: len(A[1::2])]
        return A
    if kind == "zerocols":
        U = gi.unpack(gi.bernoulli_matrix(m, n, seed), m, n)
        U[:, ::5] = 0
        U[:, 70:200] = 0
        return gi.pack(U)
    if kind == "lastrow_pivot":
        # column 0 is zero except in the last row: its pivot lies far below the
        # fast path's window
        U = gi.unpack(gi.bernoulli_matrix(m, n, seed), m, n)
        U[:, 0] = 0
        U[m - 1, 0] = 1
        return gi.pack(U)
    if kind == "identity":
        return gi.pack(np.eye(m, n, dtype=np.uint8))
    if kind == "perm":
        rng = np.random.default_rng(seed)
        U = np.zeros((m, n), dtype=np.uint8)
        cols = rng.permutation(n)[:m] if n >= m else None
        for i in range(min(m, n)):
            U[i, cols[i] if cols is not None else i] = 1
        return gi.pack(U[rng.permutation(m)])
    if kind == "zeros":
        return np.zeros((m, gi.words_for(n)), dtype=np.uint64)
    if kind == "ones":
        return gi.pack(np.ones((m, n), dtype=np.uint8))
    raise ValueError(kind)


def run_ple(h, A, m, n, ld_extra=0):
    W = gi.words_for(n)
    dA = to_dev(A, W + ld_extra)
    P = vec_dev(m)
    Q = vec_dev(min(m, n))
    r = h.ple(dA, m, n, P, Q)
    return r, to_host(dA, W), P.cpu().numpy()[:m], Q.cpu().numpy()[:min(m, n)]


def ref_ple(A, m, n):
    B = A.copy()
    r, P, Q = oracle.ple(B, m, n)
    return r, B, P, Q


def assert_ple_equal(got, want):
    r, LE, P, Q = got
    r0, LE0, P0, Q0 = want
    assert r == r0
    assert np.array_equal(P, P0)
    assert np.array_equal(Q, Q0)
    if not np.array_equal(LE, LE0):
        bad = np.argwhere(LE != LE0)
        raise AssertionError(f"L\\E differs at {len(bad)} words, first (row, word) {bad[:5].tolist()}")


SHAPES = [(1, 1), (1, 200), (200, 1), (2, 2), (63, 65), (64, 64), (65, 64), (100, 700), (700, 100),
          (257, 300), (1000, 1000), (513, 4099), (3000, 2049)]


@pytest.mark.parametrize("m,n", SHAPES)
def test_ple_dense_shapes(h, m, n):
    A = make("dense", m, n, seed=m * 7919 + n)
    assert_ple_equal(run_ple(h, A, m, n), ref_ple(A, m, n))


@pytest.mark.parametrize("kind", ["sparse", "lowrank", "zerorows", "duprows", "zerocols",
                                  "lastrow_pivot", "identity", "perm", "zeros", "ones"])
@pytest.mark.parametrize("m,n", [(300, 300), (700, 1100), (1100, 700)])
def test_ple_structured(h, kind, m, n):
    A = make(kind, m, n, seed=zlib.crc32(f"{kind}-{m}-{n}".encode()) & 0xFFFF)
    assert_ple_equal(run_ple(h, A, m, n), ref_ple(A, m, n))


def test_ple_config_2048_dense(h):
    """The 2048 x 2048 Bernoulli(1/2) workload, bit-exact against the oracle."""
    A = gi.dense_square(2048)
    assert_ple_equal(run_ple(h, A, 2048, 2048), ref_ple(A, 2048, 2048))


@pytest.mark.parametrize("ld_extra", [1, 3])
def test_ple_odd_and_padded_leading_dimension(h, ld_extra):
    m, n = 600, 900
    A = make("dense", m, n, seed=5)
    assert_ple_equal(run_ple(h, A, m, n, ld_extra=ld_extra), ref_ple(A, m, n))


def test_block_wide_panel_is_used_and_exact(h):
    h.reset_stats()
    m, n = 2000, 300
    A = make("lastrow_pivot", m, n, seed=11)
    assert_ple_equal(run_ple(h, A, m, n), ref_ple(A, m, n))
    assert h.stats()["panel_fallbacks"] >= 1


def test_ple_repeated_calls_reuse_workspace(h):
    for m, n in [(900, 900), (100, 2000), (900, 900)]:
        A = make("dense", m, n, seed=m + n)
        assert_ple_equal(run_ple(h, A, m, n), ref_ple(A, m, n))


# ----------------------------------------------------------------------- RREF

@pytest.mark.parametrize("kind", ["dense", "sparse", "lowrank", "zerocols", "lastrow_pivot"])
@pytest.mark.parametrize("m,n", [(1, 1), (65, 63), (300, 700), (700, 300), (1000, 1000)])
def test_rref(h, kind, m, n):
    A = make(kind, m, n, seed=m + 3 * n)
    W = gi.words_for(n)
    dA = to_dev(A)
    Q = vec_dev(min(m, n))
    r = h.rref(dA, m, n, Q)
    R0 = A.copy()
    r0, Q0 = oracle.rref(R0, m, n)
    assert r == r0
    assert np.array_equal(Q.cpu().numpy()[:min(m, n)], Q0)
    assert np.array_equal(to_host(dA, W), R0)


def test_rref_config_2048(h):
    A = gi.dense_square(2048)
    dA = to_dev(A)
    Q = vec_dev(2048)
    r = h.rref(dA, 2048, 2048, Q)
    R0 = A.copy()
    r0, Q0 = oracle.rref(R0, 2048, 2048)
    assert r == r0 and np.array_equal(Q.cpu().numpy(), Q0)
    assert np.array_equal(to_host(dA), R0)


# -------------------------------------------------------------------- product

@pytest.mark.parametrize("m,k,n", [(1, 1, 1), (100, 70, 130), (1000, 1000, 1000), (513, 2049, 300),
                                   (64, 0, 64), (300, 65, 1)])
@pytest.mark.parametrize("accumulate", [False, True])
def test_mul(h, m, k, n, accumulate):
    A = gi.bernoulli_matrix(m, k, 1) if k else np.zeros((m, 1), np.uint64)
    B = gi.bernoulli_matrix(k, n, 2) if k else np.zeros((1, gi.words_for(n)), np.uint64)
    C0 = gi.bernoulli_matrix(m, n, 3)
    dC = to_dev(C0)
    h.mul(dC, to_dev(A), to_dev(B), m, k, n, accumulate=accumulate)
    want = C0.copy() if accumulate else np.zeros_like(C0)
    if k:
        oracle.mul(A, B, m, k, n, C=want, accumulate=accumulate)
    assert np.array_equal(to_host(dC), want)


# ---------------------------------------------------------------------- solve

@pytest.mark.parametrize("n", [1, 5, 64, 100, 300, 1000])
@pytest.mark.parametrize("nrhs", [1, 7, 64, 65])
@pytest.mark.parametrize("kind", ["random", "singular_consistent", "singular_inconsistent"])
def test_solve(h, n, nrhs, kind):
    A = gi.bernoulli_matrix(n, n, n + nrhs)
    if kind != "random" and n > 1:
        U = gi.unpack(A, n, n)
        U[-1] = U[0] ^ U[n // 2]
        A = gi.pack(U)
    if kind == "singular_consistent":
        X = gi.bernoulli_matrix(n, nrhs, 99)
        B = oracle.mul(A, X, n, n, nrhs)
    else:
        B = gi.bernoulli_matrix(n, nrhs, 77)
    A0, B0 = A.copy(), B.copy()
    st0, r0 = oracle.solve(A0, B0, n, nrhs)
    dA, dB = to_dev(A), to_dev(B)
    st = h.solve(dA, dB, n, nrhs)
    assert st == st0
    assert np.array_equal(to_host(dA, gi.words_for(n)), A0)
    if st != oracle.SOLVE_INCONSISTENT:
        assert np.array_equal(to_host(dB, gi.words_for(nrhs)), B0)


# -------------------------------------------------------------------- batched

def _batched_check(h, mats):
    """Run gf2_ple_batched on [(A, m, n, ld_extra)] and compare each with the oracle."""
    import concurrent.futures as cf
    import torch
    items = []
    for A, m, n, extra in mats:
        dA = to_dev(A, gi.words_for(n) + extra) if m > 0 else torch.zeros((1, 1), dtype=torch.int64,
                                                                           device="cuda")
        items.append((dA, m, n, vec_dev(m), vec_dev(min(m, n)), vec_dev(1)))
    h.ple_batched(items)
    torch.cuda.synchronize()
    with cf.ThreadPoolExecutor(max_workers=16) as ex:
        refs = list(ex.map(lambda t: ref_ple_1(t[0], t[1], t[2]), mats))
    for (dA, m, n, P, Q, rk), want in zip(items, refs):
        got = (int(rk.cpu()[0]), to_host(dA, gi.words_for(n)) if m > 0 and n > 0 else want[1],
               P.cpu().numpy()[:m], Q.cpu().numpy()[:min(m, n)])
        assert_ple_equal(got, want)


def ref_ple_1(A, m, n):
    B = A.copy()
    r, P, Q = oracle.ple(B, m, n, threads=1)
    return r, B, P, Q


def test_ple_batched_matches_oracle_small(h):
    specs = gi.batch_recipe(count=24)
    _batched_check(h, [(gi.batch_matrix(sp), sp["m"], sp["n"], 0) for sp in specs])


def test_ple_batched_workload_4096(h):
    """The batched workload: 4096 matrices, sides uniform in 64..1024, 25% with
    10% of rows zeroed; every result bit-exact against the oracle."""
    specs = gi.batch_recipe(count=4096)
    _batched_check(h, [(gi.batch_matrix(sp), sp["m"], sp["n"], 0) for sp in specs])


def test_ple_batched_mixed_sizes_and_edges(h):
    mats = [(make("dense", 5000, 300, 1), 5000, 300, 0),        # beyond the batched kernel
            (make("lastrow_pivot", 1500, 200, 2), 1500, 200, 0),  # block-wide panel inside a CTA
            (make("sparse", 700, 900, 3), 700, 900, 1),          # odd leading dimension
            (make("dense", 1, 1, 4), 1, 1, 0),
            (make("zeros", 64, 64, 5), 64, 64, 0),
            (np.zeros((3, 1), np.uint64), 3, 0, 0),              # no columns
            (np.zeros((0, 1), np.uint64), 0, 5, 0)]              # no rows
    _batched_check(h, mats)


# ------------------------------------------------------------ host-buffer API

def test_host_buffer_forms(h):
    m, n = 777, 1500
    A = make("dense", m, n, 4)
    A1 = A.copy()
    r, P, Q = h.ple_host(A1, m, n)
    assert_ple_equal((r, A1, P, Q), ref_ple(A, m, n))
    A2 = A.copy()
    Qh = np.zeros(min(m, n), dtype=np.int64)
    r2 = h.rref_host(A2, m, n, Qh)
    R0 = A.copy()
    r0, Q0 = oracle.rref(R0, m, n)
    assert r2 == r0 and np.array_equal(Qh, Q0) and np.array_equal(A2, R0)


def test_empty_inputs(h):
    import torch
    dA = torch.zeros((1, 1), dtype=torch.int64, device="cuda")
    P, Q = vec_dev(4), vec_dev(1)
    assert h.ple(dA, 0, 10, P, Q) == 0
    dA4 = torch.zeros((4, 1), dtype=torch.int64, device="cuda")
    assert h.ple(dA4, 4, 0, P, Q) == 0
    assert P.cpu().numpy()[:4].tolist() == [0, 1, 2, 3]
    assert h.rref(dA4, 4, 0, Q) == 0
