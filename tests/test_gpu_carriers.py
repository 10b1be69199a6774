"""Tensor-core carriers of a GF(2) product: every carrier's AND-count product
of random bit matrices equals popcount(a & b) computed on the host (the
integer product behind Section 3.3's block multiplication), and the rate
runs keep their counts exact."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _popc_counts(a, b, words):
    """counts[i, j] = popcount of (row i AND column j) over `words` 64-bit words."""
    out = np.zeros((a.shape[0] // words, b.shape[0] // words), dtype=np.int64)
    A = a.reshape(-1, words)
    B = b.reshape(-1, words)
    for w in range(words):
        x = A[:, w][:, None] & B[:, w][None, :]
        for s in range(0, 64, 8):
            out += np.array([bin(v).count("1") for v in range(256)], dtype=np.int64)[((x >> np.uint64(s)) & np.uint64(255)).astype(np.int64)]
    return out


@pytest.mark.parametrize("carrier,rows,cols,words", [(1, 16, 8, 4), (8, 128, 256, 1), (4, 128, 256, 1),
                                                     (16, 128, 256, 1)])
@pytest.mark.parametrize("seed", [0, 1])
def test_carrier_counts_exact(carrier, rows, cols, words, seed):
    import torch
    import paper_1111_6549_gb300 as g
    rng = np.random.default_rng(1000 + seed * 10 + carrier)
    a = rng.integers(0, 2**63, size=rows * words, dtype=np.uint64) ^ (rng.integers(0, 2, size=rows * words, dtype=np.uint64) << np.uint64(63))
    b = rng.integers(0, 2**63, size=cols * words, dtype=np.uint64) ^ (rng.integers(0, 2, size=cols * words, dtype=np.uint64) << np.uint64(63))
    if seed == 1:
        a[:words] = 0                     # an all-zero row and an all-ones column
        b[:words] = np.uint64(2**64 - 1)
    da = torch.from_numpy(a.view(np.int64)).cuda()
    db = torch.from_numpy(b.view(np.int64)).cuda()
    dc = torch.full((rows * cols,), -1, dtype=torch.int32, device="cuda")
    g.carrier_check(carrier, da, db, dc)
    got = dc.cpu().numpy().reshape(rows, cols)
    want = _popc_counts(a, b, words)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("carrier,per", [(1, 256), (8, 64), (4, 64), (16, 64)])
def test_carrier_rate_counts(carrier, per):
    import paper_1111_6549_gb300 as g
    rate, cnt = g.carrier_rate(carrier, 64)
    assert rate > 0
    assert cnt == 64 * per
