"""The sparse regime of Section 4's Figure: 10000 x 10000 matrices with
exactly w nonzeros per row (w = 1 .. 200).  Very sparse inputs are rank
deficient with pivots scattered far below the panel window, so they exercise
the block-wide pivot search and the all-zero-stripe skip; every output is
bit-exact against the oracle."""
import numpy as np
import pytest

import gf2inputs as gi
import oracle
from tests.gpu_util import to_dev, to_host, vec_dev
from tests.test_gpu_parity import assert_ple_equal, ref_ple, run_ple

pytestmark = pytest.mark.gpu

N = 10000


@pytest.fixture(scope="module")
def h():
    import paper_1111_6549_gb300 as g
    return g.Handle()


@pytest.mark.parametrize("w", [1, 2, 10, 40, 200])
def test_sparse_rows_ple_and_rref(h, w):
    A = gi.row_weight_matrix(N, N, w)
    assert_ple_equal(run_ple(h, A, N, N), ref_ple(A, N, N))
    dR = to_dev(A)
    Q = vec_dev(N)
    r = h.rref(dR, N, N, Q)
    R0 = A.copy()
    r0, Q0 = oracle.rref(R0, N, N)
    assert r == r0 and np.array_equal(Q.cpu().numpy()[:r0], Q0[:r0])
    assert np.array_equal(to_host(dR, gi.words_for(N)), R0)
