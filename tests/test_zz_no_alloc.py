"""gf2_ple_noalloc against gf2_ple.

gf2_ple_noalloc serves callers that cannot allocate device memory: it takes
all of its scratch from a fixed array inside the library instead of a
handle's workspace.  Its results must be the ones gf2_ple gives, bit for
bit, on consecutive calls (the shared array keeps the previous call's
contents, so the second call checks that everything is re-initialised).
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import gf2inputs as gi
from tests.gpu_util import to_dev, to_host, vec_dev

pytestmark = pytest.mark.gpu


def _ple_existing(h, A, m, n):
    dA = to_dev(A)
    P, Q = vec_dev(m), vec_dev(min(m, n))
    r = h.ple(dA, m, n, P, Q)
    return r, to_host(dA, gi.words_for(n)), P.cpu().numpy()[:m], Q.cpu().numpy()[:min(m, n)]


def _ple_noalloc(A, m, n, ld=None, offset=0):
    """Run gf2_ple_noalloc on a device copy of A with ld words per row, the
    matrix starting `offset` words into its buffer (offset 1: a base that is
    only 8-byte aligned)."""
    import torch
    import paper_1111_6549_gb300 as g
    w = gi.words_for(n)
    ld = w if ld is None else ld
    flat = np.zeros(offset + m * ld + 1, dtype=np.uint64)
    flat[offset:offset + m * ld].reshape(m, ld)[:, :w] = A
    buf = torch.from_numpy(flat.view(np.int64)).cuda()
    dA = buf[offset:offset + m * ld].view(m, ld)
    P, Q = vec_dev(m), vec_dev(min(m, n))
    r = g.ple_noalloc(dA, m, n, P, Q)
    out = dA.cpu().numpy().view(np.uint64)[:, :w]
    return r, np.ascontiguousarray(out), P.cpu().numpy()[:m], Q.cpu().numpy()[:min(m, n)]


def test_noalloc_matches_ple_on_consecutive_calls():
    import paper_1111_6549_gb300 as g
    h = g.Handle()
    cases = [("dense", 4096, 4096), ("lowrank", 3000, 1000), ("dense", 700, 2500)]
    for kind, m, n in cases:
        if kind == "dense":
            A = gi.bernoulli_matrix(m, n, seed=m + n)
        else:
            U = gi.unpack(gi.bernoulli_matrix(m, n, seed=7), m, n)
            U[1::2] = U[0::2][: len(U[1::2])]          # every odd row repeats the one above
            A = gi.pack(U)
        want = _ple_existing(h, A, m, n)
        for _ in range(2):                              # two calls in a row
            got = _ple_noalloc(A, m, n)
            assert got[0] == want[0]
            assert np.array_equal(got[2], want[2])
            assert np.array_equal(got[3], want[3])
            assert np.array_equal(got[1], want[1])


def test_noalloc_matches_the_oracle_with_odd_and_padded_rows():
    """Against the CPU oracle directly, with leading dimensions that send the
    update through its word-by-word form: an odd ld (n = 960, 15 words) and a
    padded ld with a base that is only 8-byte aligned."""
    import oracle
    for m, n, ld, offset in [(960, 960, 15, 0), (1000, 700, 12, 1), (513, 1500, 24, 0)]:
        A = gi.bernoulli_matrix(m, n, seed=3 * m + n)
        ref = A.copy()
        r0, P0, Q0 = oracle.ple(ref, m, n)
        for _ in range(2):
            r, out, P, Q = _ple_noalloc(A, m, n, ld, offset)
            assert r == r0
            assert np.array_equal(P, P0)
            assert np.array_equal(Q, Q0)
            assert np.array_equal(out, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_1111_6549_gb300 as g
    L = g.load()
    f = L.gf2_ple_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]
    rank = ctypes.c_int64(-1)
    A = vec_dev(8)
    assert f(A.data_ptr(), 4097, 64, 1, A.data_ptr(), A.data_ptr(), ctypes.byref(rank), None) == 1
    assert f(A.data_ptr(), 64, 4097, 65, A.data_ptr(), A.data_ptr(), ctypes.byref(rank), None) == 1


def test_noalloc_refuses_a_capturing_stream():
    """The call synchronises its stream, so it must not be captured: on a
    capturing stream it returns GF2_EINVAL before enqueueing anything."""
    import torch
    import paper_1111_6549_gb300 as g
    m = n = 256
    A = gi.bernoulli_matrix(m, n, seed=11)
    _ple_noalloc(A, m, n)                       # first call on the device: address lookup
    L = g.load()
    f = L.gf2_ple_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]
    dA = to_dev(A)
    P, Q = vec_dev(m), vec_dev(n)
    rank = ctypes.c_int64(-1)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        rc = f(dA.data_ptr(), m, n, gi.words_for(n), P.data_ptr(), Q.data_ptr(), ctypes.byref(rank),
               ctypes.c_void_p(s.cuda_stream))
        P.add_(0)                               # keep the captured graph non-empty
    assert rc == 1                              # GF2_EINVAL
    del graph
