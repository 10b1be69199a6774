"""Failure detection without a GPU fault: a bounded device-side wait that can
only expire (an mbarrier nothing arrives on) is reported as GF2_ETIMEOUT, and
the same handle keeps working afterwards."""
import numpy as np
import pytest

import gf2inputs as gi
import oracle
from tests.gpu_util import to_dev, to_host, vec_dev

pytestmark = pytest.mark.gpu


def test_expired_wait_is_reported_and_handle_stays_usable():
    import paper_1111_6549_gb300 as g
    h = g.Handle()
    assert h.selftest_wait(2000) == g.GF2_ETIMEOUT
    assert h.selftest_wait(0) == g.GF2_ETIMEOUT
    m, n = 500, 700
    A = gi.bernoulli_matrix(m, n, 77)
    dA = to_dev(A)
    P, Q = vec_dev(m), vec_dev(min(m, n))
    r = h.ple(dA, m, n, P, Q)
    LE = A.copy()
    r0, P0, Q0 = oracle.ple(LE, m, n)
    assert r == r0 and np.array_equal(to_host(dA, gi.words_for(n)), LE)


def test_selftest_rejects_bad_limits():
    import paper_1111_6549_gb300 as g
    h = g.Handle()
    assert h.selftest_wait(-1) == g.GF2_EINVAL
    assert h.selftest_wait(10**7) == g.GF2_EINVAL
