"""The own tensor-core GEMM of the GF(2) product (tcgen05 kind::mxf4, TMA-fed,
parities taken from tensor memory): C = A B and C ^= A B bit-exact against
the oracle's product (Section 3.3's block multiplication), with every size
ragged against the 256 x 192 output tiles, the 256-value inner stages and the
64-bit words, and with leading dimensions padded past the row width."""
import numpy as np
import pytest

import gf2inputs as gi
import oracle
from tests.gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    import paper_1111_6549_gb300 as g
    hh = g.Handle()
    hh.set_option(g.OPT_MUL_GEMM_FORMAT, 0)
    hh.set_option(g.OPT_MUL_GEMM_MIN_K, 1)      # every product through the GEMM
    return hh


@pytest.mark.parametrize("m,k,n", [(256, 256, 192), (1, 1, 1), (300, 70, 300), (257, 4097, 193),
                                   (1000, 5000, 777), (513, 2049, 4100), (2048, 8192, 2048),
                                   (100, 300, 64), (4096, 1000, 385)])
@pytest.mark.parametrize("accumulate", [False, True])
def test_gemm_f4_mul(h, m, k, n, accumulate):
    A = gi.bernoulli_matrix(m, k, 31 + m)
    B = gi.bernoulli_matrix(k, n, 37 + n)
    C0 = gi.bernoulli_matrix(m, n, 41 + k)
    pad = 3 if m % 2 else 0                        # odd, padded leading dimensions on some cases
    dC = to_dev(C0, gi.words_for(n) + pad)
    h.mul(dC, to_dev(A, gi.words_for(k) + pad), to_dev(B, gi.words_for(n) + pad), m, k, n,
          accumulate=accumulate)
    want = C0.copy() if accumulate else np.zeros_like(C0)
    oracle.mul(A, B, m, k, n, C=want, accumulate=accumulate)
    assert np.array_equal(to_host(dC, gi.words_for(n)), want)


def test_gemm_f4_structured(h):
    """All-ones operands give counts equal to k (parity k mod 2 everywhere),
    identity gives A back: the two ends of the count range."""
    m, k, n = 512, 4096 + 64, 384
    ones_a = np.full((m, gi.words_for(k)), np.uint64(2**64 - 1), dtype=np.uint64)
    ones_b = np.full((k, gi.words_for(n)), np.uint64(2**64 - 1), dtype=np.uint64)
    dC = to_dev(np.zeros((m, gi.words_for(n)), np.uint64))
    h.mul(dC, to_dev(ones_a), to_dev(ones_b), m, k, n)
    assert not to_host(dC).any()                   # k even: every parity 0
    k2 = k + 1
    ones_a2 = gi.bernoulli_matrix(m, k2, 1) | np.uint64(2**64 - 1)
    ones_a2 = gi.pack(gi.unpack(ones_a2, m, k2))
    ones_b2 = gi.pack(gi.unpack(np.full((k2, gi.words_for(n)), np.uint64(2**64 - 1), dtype=np.uint64), k2, n))
    h.mul(dC, to_dev(ones_a2), to_dev(ones_b2), m, k2, n)
    want = gi.pack(np.ones((m, n), dtype=np.uint8))
    assert np.array_equal(to_host(dC), want)       # k odd: every parity 1
    eye = gi.pack(np.eye(n, dtype=np.uint8))
    A = gi.bernoulli_matrix(m, n, 5)
    h.mul(dC, to_dev(A), to_dev(eye), m, n, n)
    assert np.array_equal(to_host(dC), A)


@pytest.mark.parametrize("level", [1, 3, 5])
def test_gemm_stats_count_flops(level):
    """Profiling levels 1 and 5 time every GEMM launch (5 nothing else), level
    3 none: the statistics carry the launches, the event time and 2 m k n of
    the timed products and of all of them."""
    import paper_1111_6549_gb300 as g
    hh = g.Handle()
    hh.set_option(g.OPT_MUL_GEMM_MIN_K, 1)
    m, k, n = 1000, 3000, 700
    A = gi.bernoulli_matrix(m, k, 3)
    B = gi.bernoulli_matrix(k, n, 4)
    dC = to_dev(np.zeros((m, gi.words_for(n)), np.uint64))
    hh.reset_stats()
    hh.set_profiling(level)
    hh.mul(dC, to_dev(A), to_dev(B), m, k, n)
    st = hh.stats()
    hh.set_profiling(0)
    assert st["gemm_launches"] >= 1 and st["gemm_flops_all"] == 2.0 * m * k * n
    if level in (1, 5):
        assert st["gemm_timed_launches"] == st["gemm_launches"]
        assert st["gemm_flops"] == 2.0 * m * k * n and st["gemm_ms"] > 0.0
    else:
        assert st["gemm_timed_launches"] == 0 and st["gemm_flops"] == 0.0
    if level == 5:
        assert st["update_timed_launches"] == 0 and st["other_ms"] == 0.0
    assert np.array_equal(to_host(dC, gi.words_for(n)), oracle.mul(A, B, m, k, n))
