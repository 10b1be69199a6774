"""The continuous-batching solve server (gf2_server_*).

Jobs submitted together overlap on the device; every job's status and
solution must be the same as when it runs alone (gf2_solve through a handle)
and, where the oracle is fast, the same as the oracle's.
"""
import numpy as np
import pytest

import gf2inputs as gi
import oracle
from tests.gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


def _jobs(count, seed=0, max_n=6000):
    st = gi.Stream(gi.BASE_SEED + 40 + seed)
    out = []
    for j in range(count):
        n = [st.randint(1, 200), st.randint(200, 1500), st.randint(1500, max_n)][j % 3]
        nrhs = st.randint(1, 64)
        A = gi.bernoulli_matrix(n, n, 1000 + j)
        kind = j % 4
        if kind >= 2 and n > 2:                    # singular
            U = gi.unpack(A, n, n)
            U[-1] = U[0] ^ U[1]
            A = gi.pack(U)
        if kind == 2:                              # consistent right-hand side
            B = oracle.mul(A, gi.bernoulli_matrix(n, nrhs, 2000 + j), n, n, nrhs)
        else:
            B = gi.bernoulli_matrix(n, nrhs, 3000 + j)
        out.append((j, A, n, B, nrhs))
    return out


def _alone(h, A, n, B, nrhs):
    dA, dB = to_dev(A), to_dev(B)
    st = h.solve(dA, dB, n, nrhs)
    return st, to_host(dB, gi.words_for(nrhs))


def _serve(jobs, slots, budget=0):
    import paper_1111_6549_gb300 as g
    srv = g.Server(slots=slots, max_n=max(n for _, _, n, _, _ in jobs), max_nrhs=64,
                   hbm_budget_bytes=budget)
    X = {}
    keep = []
    for j, A, n, B, nrhs in jobs:
        Ah, Bh = np.ascontiguousarray(A), np.ascontiguousarray(B)
        Xh = np.zeros((n, gi.words_for(nrhs)), dtype=np.uint64)
        keep.append((Ah, Bh, Xh))
        X[j] = Xh
        srv.submit(j, Ah, n, Bh, nrhs, Xh)
    srv.drain()
    res = {r[0]: r for r in srv.poll(len(jobs) + 8)}
    srv.close()
    return res, X


def test_server_results_same_alone_and_in_the_mix():
    import paper_1111_6549_gb300 as g
    h = g.Handle()
    jobs = _jobs(24)
    res, X = _serve(jobs, slots=4)
    assert sorted(res) == [j for j, *_ in jobs]
    overlapped = 0
    for j, A, n, B, nrhs in jobs:
        _, status, err, t_sub, t_start, t_done = res[j]
        assert err == 0
        st_alone, X_alone = _alone(h, A, n, B, nrhs)
        assert status == st_alone
        if status != g.SOLVE_INCONSISTENT:
            assert np.array_equal(X[j], X_alone)
        if n <= 2000:
            A0, B0 = A.copy(), B.copy()
            st0, _ = oracle.solve(A0, B0, n, nrhs)
            assert status == st0
            if st0 != oracle.SOLVE_INCONSISTENT:
                assert np.array_equal(X[j], B0)
        overlapped += sum(1 for k in res if k != j and res[k][4] < t_done and res[k][5] > t_start)
    assert overlapped > 0          # several jobs were on the device at the same time


def test_server_budget_admits_one_at_a_time():
    """With a budget smaller than any two jobs, jobs run one after another and
    are still all correct."""
    import paper_1111_6549_gb300 as g
    h = g.Handle()
    jobs = _jobs(6, seed=1, max_n=2500)
    res, X = _serve(jobs, slots=4, budget=1)
    spans = sorted((res[j][4], res[j][5]) for j, *_ in jobs)
    for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
        assert s1 >= e0 - 1e-4     # no overlap (completion is seen before the next start)
    for j, A, n, B, nrhs in jobs:
        st_alone, X_alone = _alone(h, A, n, B, nrhs)
        assert res[j][1] == st_alone
        if st_alone != g.SOLVE_INCONSISTENT:
            assert np.array_equal(X[j], X_alone)
