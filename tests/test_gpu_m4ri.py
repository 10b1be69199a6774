"""M4RI (Algorithm 8): the RREF in one sweep, bit-exact against the oracle's
RREF (unique by Section 2), with the same rank and pivot columns."""
import numpy as np
import pytest

import gf2inputs as gi
import oracle
from tests.gpu_util import to_dev, to_host, vec_dev
from tests.test_gpu_parity import make

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    import paper_1111_6549_gb300 as g
    return g.Handle()


def check_m4ri(h, A, m, n, ld_extra=0):
    W = gi.words_for(n)
    dA = to_dev(A, W + ld_extra)
    Q = vec_dev(max(min(m, n), 1))
    r = h.rref_m4ri(dA, m, n, Q)
    R0 = A.copy()
    r0, Q0 = oracle.rref(R0, m, n)
    assert r == r0
    assert np.array_equal(Q.cpu().numpy()[:min(m, n)], Q0)
    got = to_host(dA, W)
    if not np.array_equal(got, R0):
        bad = np.argwhere(got != R0)
        raise AssertionError(f"RREF differs at {len(bad)} words, first {bad[:5].tolist()}")


SHAPES = [(1, 1), (1, 200), (200, 1), (2, 2), (63, 65), (64, 64), (65, 64), (100, 700), (700, 100),
          (257, 300), (1000, 1000), (513, 4099), (3000, 2049), (2048, 2048)]


@pytest.mark.parametrize("m,n", SHAPES)
def test_m4ri_dense_shapes(h, m, n):
    check_m4ri(h, make("dense", m, n, seed=m * 31 + n), m, n)


@pytest.mark.parametrize("kind", ["sparse", "lowrank", "zerorows", "duprows", "zerocols", "lastrow_pivot",
                                  "identity", "perm", "zeros", "ones"])
def test_m4ri_structured(h, kind):
    m, n = 900, 1300
    check_m4ri(h, make(kind, m, n, seed=5), m, n)


def test_m4ri_odd_leading_dimension(h):
    check_m4ri(h, make("dense", 777, 1500, seed=2), 777, 1500, ld_extra=1)
    check_m4ri(h, make("lowrank", 1200, 800, seed=3), 1200, 800, ld_extra=3)


@pytest.mark.parametrize("w", [1, 40])
def test_m4ri_sparse_rows(h, w):
    A = gi.row_weight_matrix(10000, 10000, w)
    check_m4ri(h, A, 10000, 10000)


def test_m4ri_structured_rank(h):
    X, Y = gi.structured_factors(m=2048, k=512, n=4096)
    A = oracle.mul(X, Y, 2048, 512, 4096)
    check_m4ri(h, A, 2048, 4096)
