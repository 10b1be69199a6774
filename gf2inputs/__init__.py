"""Seeded synthetic inputs for the GF(2) elimination workloads.

This module is shared by the CPU oracle's tests and by the CUDA path's tests
and benchmark.  It holds no GF(2) linear algebra: only pseudo-random bit
generation, bit packing and workload size recipes.

Bit layout (used everywhere in this repository): a GF(2) matrix with ``m`` rows
and ``n`` columns is stored row-major as ``uint64`` words, ``ld`` words per row
(``ld >= ceil(n/64)``).  Column ``j`` is bit ``j % 64`` (LSB = lowest column) of
word ``j // 64``.  Bits at columns ``>= n`` (padding) are zero.

Random numbers: every row ``i`` of a matrix drawn with seed ``s`` has its own
xoshiro256** stream (Blackman & Vigna, 2018), whose 256-bit state is four
consecutive outputs of splitmix64 (Steele, Lea & Flood, 2014) started at
``x = s + i * 0x632BE59BD9B4E019 (mod 2^64)``.  Word ``w`` of row ``i`` is the
``w``-th output of that stream (Bernoulli(1/2) bits); a Bernoulli(1/16) word is
the AND of four consecutive outputs.  The streams are evaluated vectorised over
rows with numpy, so a 65536 x 65536 matrix (512 MiB) takes about a second.
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = 0x9E3779B97F4A7C15
_ROW_STRIDE = 0x632BE59BD9B4E019
BASE_SEED = 0x11116549  # per-workload seeds are BASE_SEED + workload index


def words_for(n: int) -> int:
    """Number of 64-bit words holding ``n`` bits."""
    return (n + 63) // 64


def _u64(x) -> np.ndarray:
    return np.asarray(x, dtype=np.uint64)


def _rotl(x: np.ndarray, k: int) -> np.ndarray:
    return (x << np.uint64(k)) | (x >> np.uint64(64 - k))


def _splitmix64_next(x: np.ndarray):
    """One splitmix64 step on an array of states; returns (new_state, output)."""
    x = x + np.uint64(_GOLDEN)
    z = x
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return x, z ^ (z >> np.uint64(31))


class RowStreams:
    """Independent xoshiro256** streams, one per row, advanced in lock step."""

    def __init__(self, seed: int, rows: int, row0: int = 0):
        idx = np.arange(row0, row0 + rows, dtype=np.uint64)
        with np.errstate(over="ignore"):
            x = _u64(seed & 0xFFFFFFFFFFFFFFFF) + idx * np.uint64(_ROW_STRIDE)
            s = []
            for _ in range(4):
                x, out = _splitmix64_next(x)
                s.append(out)
        self.s0, self.s1, self.s2, self.s3 = s

    def next(self) -> np.ndarray:
        with np.errstate(over="ignore"):
            s0, s1, s2, s3 = self.s0, self.s1, self.s2, self.s3
            result = _rotl(s1 * np.uint64(5), 7) * np.uint64(9)
            t = s1 << np.uint64(17)
            s2 = s2 ^ s0
            s3 = s3 ^ s1
            s1 = s1 ^ s2
            s0 = s0 ^ s3
            s2 = s2 ^ t
            s3 = _rotl(s3, 45)
            self.s0, self.s1, self.s2, self.s3 = s0, s1, s2, s3
        return result


class Stream:
    """A single scalar xoshiro256** stream (used for sizes and choices)."""

    def __init__(self, seed: int):
        self._rs = RowStreams(seed, 1)

    def u64(self) -> int:
        return int(self._rs.next()[0])

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.u64() >> 11) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive), by rejection."""
        span = hi - lo + 1
        limit = (1 << 64) - ((1 << 64) % span)
        while True:
            v = self.u64()
            if v < limit:
                return lo + v % span


def pad_mask(n: int) -> int:
    """Mask of the valid bits in the last word of an n-column row."""
    rem = n % 64
    return 0xFFFFFFFFFFFFFFFF if rem == 0 else (1 << rem) - 1


def bernoulli_matrix(m: int, n: int, seed: int, ld: int | None = None,
                     density_log2: int = 1, row0: int = 0) -> np.ndarray:
    """m x n matrix of i.i.d. Bernoulli(2**-density_log2) bits, packed.

    ``density_log2 = 1`` gives Bernoulli(1/2) (one stream word per matrix
    word); ``density_log2 = 4`` gives Bernoulli(1/16) (AND of four words).
    ``row0`` selects rows ``row0 .. row0+m-1`` of the same seeded matrix, so a
    row block of a large matrix can be regenerated without the rest.
    Returns an ``(m, ld)`` uint64 array; padding words/bits are zero.
    """
    w = words_for(n)
    ld = w if ld is None else ld
    if ld < w:
        raise ValueError("ld must be >= ceil(n/64)")
    out = np.zeros((m, ld), dtype=np.uint64)
    if m == 0 or n == 0:
        return out
    rs = RowStreams(seed, m, row0)
    for k in range(w):
        v = rs.next()
        for _ in range(density_log2 - 1):
            v = v & rs.next()
        out[:, k] = v
    out[:, w - 1] &= np.uint64(pad_mask(n))
    return out


def unpack(A: np.ndarray, m: int, n: int) -> np.ndarray:
    """Packed (m, ld) uint64 -> (m, n) uint8 of 0/1 (column j = bit j%64 of word j//64)."""
    if m == 0 or n == 0:
        return np.zeros((m, n), dtype=np.uint8)
    w = words_for(n)
    b = A[:m, :w].astype("<u8").view(np.uint8).reshape(m, w * 8)
    bits = np.unpackbits(b, axis=1, bitorder="little")
    return bits[:, :n].copy()


def pack(U: np.ndarray, ld: int | None = None) -> np.ndarray:
    """(m, n) 0/1 array -> packed (m, ld) uint64 with the repository bit layout."""
    U = np.asarray(U, dtype=np.uint8)
    m, n = U.shape
    w = words_for(n)
    ld = w if ld is None else ld
    out = np.zeros((m, ld), dtype=np.uint64)
    if m == 0 or n == 0:
        return out
    padded = np.zeros((m, w * 64), dtype=np.uint8)
    padded[:, :n] = U & 1
    by = np.packbits(padded, axis=1, bitorder="little")
    out[:, :w] = by.view("<u8").reshape(m, w)
    return out


def zero_rows(A: np.ndarray, rows) -> None:
    """Zero the given rows in place (used for the rank-deficient batch recipe)."""
    A[np.asarray(rows, dtype=np.int64), :] = 0


# --------------------------------------------------------------------------
# Workload recipes (shapes and distributions of the paper's workloads)
# --------------------------------------------------------------------------

def dense_square(n: int, seed: int = BASE_SEED + 1) -> np.ndarray:
    """Dense random n x n matrix, Bernoulli(1/2) bits (Section 5, Table 2 workloads)."""
    return bernoulli_matrix(n, n, seed)


def sparse_square(n: int, seed: int = BASE_SEED + 2) -> np.ndarray:
    """n x n matrix with Bernoulli(1/16) bits (the moderately sparse regime of Section 4)."""
    return bernoulli_matrix(n, n, seed, density_log2=4)


def row_weight_matrix(m: int, n: int, w: int, seed: int = BASE_SEED + 5) -> np.ndarray:
    """m x n matrix with exactly w ones per row at uniformly random distinct
    columns (the sparse workloads of Section 4's Figure: 10000 x 10000 with
    1..200 nonzeros per row).  Floyd's sampling, one draw per row and step."""
    assert 0 <= w <= n
    W = words_for(n)
    A = np.zeros((m, W), dtype=np.uint64)
    rs = RowStreams(seed, m)
    rows = np.arange(m)
    one = np.uint64(1)
    for j in range(n - w, n):
        u = rs.next()
        t = (u % np.uint64(j + 1)).astype(np.int64)
        taken = (A[rows, t >> 6] >> (t & 63).astype(np.uint64)) & one
        c = np.where(taken == one, j, t)
        A[rows, c >> 6] |= one << (c & 63).astype(np.uint64)
    return A


def structured_factors(m: int = 16384, k: int = 8192, n: int = 32768,
                       seed: int = BASE_SEED + 2):
    """The two Bernoulli(1/2) factors X (m x k) and Y (k x n) of the rank-k workload.

    The workload matrix is their GF(2) product, which the caller forms with
    the multiplication under test (the product is linear algebra and does not
    belong in this module).
    """
    return bernoulli_matrix(m, k, seed), bernoulli_matrix(k, n, seed + 1)


def batch_recipe(count: int = 4096, lo: int = 64, hi: int = 1024,
                 seed: int = BASE_SEED + 3, deficient_frac: float = 0.25,
                 zero_frac: float = 0.10):
    """Sizes and row-zeroing choices of the batched workload.

    Returns a list of dicts ``{m, n, seed, zero_rows}``: matrix ``b`` has
    ``m, n ~ U{lo..hi}``, Bernoulli(1/2) bits from seed ``seed + 1 + b``, and
    for a seeded 25% of matrices ``floor(0.1 m)`` distinct random rows zeroed
    after generation.
    """
    st = Stream(seed)
    out = []
    for b in range(count):
        m = st.randint(lo, hi)
        n = st.randint(lo, hi)
        zr = []
        if st.uniform() < deficient_frac:
            kz = int(math.floor(zero_frac * m))
            chosen = set()
            while len(chosen) < kz:
                chosen.add(st.randint(0, m - 1))
            zr = sorted(chosen)
        out.append({"m": m, "n": n, "seed": seed + 1 + b, "zero_rows": zr})
    return out


def batch_matrix(spec: dict) -> np.ndarray:
    """Materialise one matrix of ``batch_recipe``."""
    A = bernoulli_matrix(spec["m"], spec["n"], spec["seed"])
    if spec["zero_rows"]:
        zero_rows(A, spec["zero_rows"])
    return A


def solve_stream_recipe(count: int, rate: float, lo: int = 128, hi: int = 16384,
                        max_rhs: int = 64, seed: int = BASE_SEED + 4):
    """Arrival times and sizes of the served solve workload.

    Poisson arrivals at ``rate`` requests/s (exponential gaps), ``n =
    floor(exp(U(ln lo, ln hi)))`` (log-uniform), ``nrhs ~ U{1..max_rhs}``, A
    and B Bernoulli(1/2) from per-job seeds.
    """
    st = Stream(seed)
    t = 0.0
    jobs = []
    for j in range(count):
        t += -math.log(1.0 - st.uniform()) / rate
        n = int(math.floor(math.exp(math.log(lo) + st.uniform() * (math.log(hi) - math.log(lo)))))
        n = max(lo, min(hi, n))
        nrhs = st.randint(1, max_rhs)
        jobs.append({"t": t, "n": n, "nrhs": nrhs, "seed": seed + 1 + 2 * j})
    return jobs


def solve_job_inputs(job: dict):
    """A (n x n) and B (n x nrhs) of one served solve job."""
    n, nrhs, s = job["n"], job["nrhs"], job["seed"]
    return bernoulli_matrix(n, n, s), bernoulli_matrix(n, nrhs, s + 1)
