"""CPU oracle for dense GF(2) PLE / RREF / product / solve.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg (and its ``--impl reference`` arm) may import
this package.  It shares no code with ``paper_1111_6549_gb300`` and never
imports it.

``gf2_oracle.c`` holds the plain definitions (eager Gaussian elimination with
the paper's pivot rule); ``gf2_checks.c`` holds size-independent property
checks used where the full oracle would take minutes; ``twin.py`` is a second,
independent implementation on unpacked 0/1 arrays following the lazy
left-looking search of Algorithm 1.  See each file's header for the passages
of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = [os.path.join(_HERE, "gf2_oracle.c"), os.path.join(_HERE, "gf2_checks.c")]

SOLVE_OK, SOLVE_UNDERDETERMINED, SOLVE_INCONSISTENT = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable C, OpenMP) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SOURCES)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp] + _SOURCES
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        i64, u64p, i64p = ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p
        c_int = ctypes.c_int
        _lib.oracle_ple.argtypes = [u64p, i64, i64, i64, i64, i64, i64p, i64p, c_int]
        _lib.oracle_ple.restype = i64
        _lib.oracle_rref.argtypes = [u64p, i64, i64, i64, i64p, c_int]
        _lib.oracle_rref.restype = i64
        _lib.oracle_mul.argtypes = [u64p, i64, u64p, i64, u64p, i64, i64, i64, i64, c_int, c_int]
        _lib.oracle_mul.restype = None
        _lib.oracle_solve.argtypes = [u64p, i64, i64, u64p, i64, i64, i64p, c_int]
        _lib.oracle_solve.restype = c_int
        _lib.check_ple_structure.argtypes = [u64p, i64, i64, i64, i64p, i64p, i64]
        _lib.check_ple_structure.restype = i64
        _lib.check_pivot_rule.argtypes = [u64p, i64, i64, i64p, i64]
        _lib.check_pivot_rule.restype = i64
        _lib.check_freivalds_ple.argtypes = [u64p, i64, u64p, i64, i64, i64, i64p, i64,
                                             ctypes.c_uint64, c_int]
        _lib.check_freivalds_ple.restype = i64
        _lib.check_rref.argtypes = [u64p, i64, u64p, i64, i64, i64, i64p, i64,
                                    ctypes.c_uint64, c_int]
        _lib.check_rref.restype = i64
    return _lib


def default_threads() -> int:
    return int(os.environ.get("GF2_ORACLE_THREADS", os.cpu_count() or 1))


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _check_mat(A: np.ndarray, m: int, n: int) -> int:
    assert A.dtype == np.uint64 and A.ndim == 2 and A.shape[0] >= m
    ld = A.shape[1]
    assert ld >= (n + 63) // 64 or m == 0 or n == 0
    return ld


def ple(A: np.ndarray, m: int, n: int, npiv: int | None = None, max_pivots: int = -1,
        threads: int | None = None):
    """PLE of the packed matrix A (modified in place to L\\E).

    Returns ``(rank, P, Q)`` with P the LAPACK-style swap vector (int64[m])
    and Q the pivot columns (int64[min(m, npiv)], -1 past the rank).
    """
    ld = _check_mat(A, m, n)
    npiv = n if npiv is None else npiv
    P = np.zeros(max(m, 0), dtype=np.int64)
    Q = np.full(max(min(m, npiv), 0), -1, dtype=np.int64)
    if m == 0 or n == 0:
        P[:] = np.arange(m)
        return 0, P, Q
    r = lib().oracle_ple(_ptr(A), m, n, ld, npiv, max_pivots, _ptr(P), _ptr(Q),
                         threads or default_threads())
    if r < 0:
        raise MemoryError("oracle_ple: allocation failed")
    return int(r), P, Q


def rref(A: np.ndarray, m: int, n: int, threads: int | None = None):
    """RREF of A in place.  Returns ``(rank, Q)``."""
    ld = _check_mat(A, m, n)
    Q = np.full(max(min(m, n), 0), -1, dtype=np.int64)
    if m == 0 or n == 0:
        return 0, Q
    r = lib().oracle_rref(_ptr(A), m, n, ld, _ptr(Q), threads or default_threads())
    if r < 0:
        raise MemoryError("oracle_rref: allocation failed")
    return int(r), Q


def mul(A: np.ndarray, B: np.ndarray, m: int, k: int, n: int, C: np.ndarray | None = None,
        accumulate: bool = False, threads: int | None = None) -> np.ndarray:
    """C = A B (or C ^= A B) over GF(2); A m x k, B k x n."""
    if C is None:
        C = np.zeros((m, max((n + 63) // 64, 1)), dtype=np.uint64)
    if m == 0 or n == 0:
        return C
    lib().oracle_mul(_ptr(C), C.shape[1], _ptr(A), A.shape[1], _ptr(B), B.shape[1],
                     m, k, n, 1 if accumulate else 0, threads or default_threads())
    return C


def solve(A: np.ndarray, B: np.ndarray, n: int, nrhs: int, threads: int | None = None):
    """Solve A X = B (A n x n, B n x nrhs), in place.  Returns ``(status, rank)``."""
    rank = np.zeros(1, dtype=np.int64)
    st = lib().oracle_solve(_ptr(A), n, A.shape[1], _ptr(B), nrhs, B.shape[1], _ptr(rank),
                            threads or default_threads())
    if st < 0:
        raise MemoryError("oracle_solve: allocation failed")
    return int(st), int(rank[0])


# ---- property checks (0 = holds) -------------------------------------------

def check_ple_structure(LE, m, n, P, Q, r) -> int:
    return int(lib().check_ple_structure(_ptr(LE), m, n, LE.shape[1], _ptr(P), _ptr(Q), r))


def check_pivot_rule(LE, m, P, r) -> int:
    return int(lib().check_pivot_rule(_ptr(LE), m, LE.shape[1], _ptr(P), r))


def check_freivalds_ple(A0, LE, m, n, P, r, seed=12345, threads=None) -> int:
    return int(lib().check_freivalds_ple(_ptr(A0), A0.shape[1], _ptr(LE), LE.shape[1], m, n,
                                         _ptr(P), r, seed, threads or default_threads()))


def check_rref(R, LE, m, n, Q, r, seed=6789, threads=None) -> int:
    return int(lib().check_rref(_ptr(R), R.shape[1], _ptr(LE), LE.shape[1], m, n, _ptr(Q), r,
                                seed, threads or default_threads()))


def check_ple_all(A0, LE, m, n, P, Q, r, threads=None) -> dict:
    """All PLE properties at once; every value must be 0."""
    return {
        "structure": check_ple_structure(LE, m, n, P, Q, r),
        "pivot_rule": check_pivot_rule(LE, m, P, r),
        "freivalds": check_freivalds_ple(A0, LE, m, n, P, r, threads=threads),
    }


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
