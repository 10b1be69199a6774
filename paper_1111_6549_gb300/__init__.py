"""GB300 GF(2) dense elimination: thin Python binding of libgf2 (include/gf2.h).

Everything computes in the CUDA library; this module only marshals
arguments.  Matrices are torch ``int64`` tensors on the GPU holding raw
64-bit words (row-major, column j = bit j % 64 of word j // 64, padding bits
zero).  There is no CPU path: if the library cannot be loaded the calls raise.

Entry points (same names as the C ABI, without the ``gf2_`` prefix):
``ple``, ``ple_async``, ``rref``, ``rref_async``, ``mul``, ``solve``,
``ple_batched``, ``ple_host``, ``rref_host``, ``workspace_bytes`` and the
statistics helpers on :class:`Handle`.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = ["Handle", "GF2Error", "load", "lib_path", "SOLVE_UNIQUE", "SOLVE_UNDERDETERMINED",
           "SOLVE_INCONSISTENT", "words_for", "default_handle"]

_HERE = os.path.dirname(os.path.abspath(__file__))

GF2_OK, GF2_EINVAL, GF2_ENOMEM, GF2_ECUDA, GF2_ETIMEOUT, GF2_EINTERNAL = range(6)
(OPT_LOOKAHEAD, OPT_TC_MUL, OPT_TC_UPDATE, OPT_TMA_UPDATE, OPT_MUL_GEMM_MIN_K, OPT_PLE_BLOCK,
 OPT_MUL_GEMM_FORMAT, OPT_RREF_BLOCK, OPT_WIDE_UPDATE, OPT_NAIVE_UPDATE, OPT_PDL,
 OPT_PLE_RECURSIVE, OPT_TRSM_LEAF, OPT_RREF_LEAF, OPT_RREF_COMPACT) = (1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14,
                                                                 15)
BATCH_CLASSES, BATCH_CONFIGS = 6, 5
SOLVE_UNIQUE, SOLVE_UNDERDETERMINED, SOLVE_INCONSISTENT = 0, 1, 2
CARRIER_B1, CARRIER_FP4, CARRIER_FP8, CARRIER_NVF4 = 1, 4, 8, 16


class GF2Error(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)}")


class _Stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("update_launches", ctypes.c_int64),
                ("update_ms", ctypes.c_double), ("update_bytes", ctypes.c_double),
                ("panel_fallbacks", ctypes.c_int64), ("panel_ms", ctypes.c_double),
                ("prep_ms", ctypes.c_double), ("rref_prep_ms", ctypes.c_double),
                ("other_ms", ctypes.c_double), ("update_timed_launches", ctypes.c_int64),
                ("rref_pass_ms", ctypes.c_double), ("rref_pass_bytes", ctypes.c_double),
                ("rref_pass_launches", ctypes.c_int64), ("rref_pass_timed_launches", ctypes.c_int64),
                ("gemm_ms", ctypes.c_double), ("gemm_flops", ctypes.c_double),
                ("gemm_launches", ctypes.c_int64), ("gemm_timed_launches", ctypes.c_int64),
                ("gemm_flops_all", ctypes.c_double)]


class SolveJob(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("A", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("lda", ctypes.c_int64), ("B", ctypes.c_void_p), ("nrhs", ctypes.c_int64),
                ("ldb", ctypes.c_int64), ("X", ctypes.c_void_p), ("ldx", ctypes.c_int64)]


class SolveResult(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int), ("error", ctypes.c_int),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


class Desc(ctypes.Structure):
    """gf2_desc of the batched entry point."""
    _fields_ = [("A", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("ld_words", ctypes.c_int64), ("P", ctypes.c_void_p), ("Q", ctypes.c_void_p),
                ("rank", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    from . import build as _build
    return _build.LIB


def load():
    """Load libgf2.so, building it first (nvcc, sm_103a) when it is missing or stale."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build
        path = _build.LIB
        if not _build.up_to_date():
            path = _build.build()
        L = ctypes.CDLL(path)
        vp, i64, i32p = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int)
        i64p = ctypes.POINTER(ctypes.c_int64)
        sig = {
            "gf2_create": ([ctypes.POINTER(vp), ctypes.c_int], ctypes.c_int),
            "gf2_destroy": ([vp], ctypes.c_int),
            "gf2_set_stream": ([vp, vp], ctypes.c_int),
            "gf2_ple": ([vp, vp, i64, i64, i64, vp, vp, i64p], ctypes.c_int),
            "gf2_ple_async": ([vp, vp, i64, i64, i64, vp, vp, vp], ctypes.c_int),
            "gf2_rref": ([vp, vp, i64, i64, i64, vp, i64p], ctypes.c_int),
            "gf2_rref_async": ([vp, vp, i64, i64, i64, vp, vp], ctypes.c_int),
            "gf2_rref_m4ri": ([vp, vp, i64, i64, i64, vp, i64p], ctypes.c_int),
            "gf2_rref_m4ri_async": ([vp, vp, i64, i64, i64, vp, vp], ctypes.c_int),
            "gf2_mul": ([vp, vp, i64, vp, i64, vp, i64, i64, i64, i64, ctypes.c_int], ctypes.c_int),
            "gf2_solve": ([vp, vp, i64, i64, vp, i64, i64, i32p], ctypes.c_int),
            "gf2_ple_batched": ([vp, ctypes.POINTER(Desc), i64], ctypes.c_int),
            "gf2_workspace_bytes": ([vp, i64, i64], ctypes.c_size_t),
            "gf2_ple_host": ([vp, vp, i64, i64, i64, vp, vp, i64p], ctypes.c_int),
            "gf2_rref_host": ([vp, vp, i64, i64, i64, vp, i64p], ctypes.c_int),
            "gf2_set_profiling": ([vp, ctypes.c_int], ctypes.c_int),
            "gf2_get_stats": ([vp, ctypes.POINTER(_Stats)], ctypes.c_int),
            "gf2_reset_stats": ([vp], ctypes.c_int),
            "gf2_strerror": ([ctypes.c_int], ctypes.c_char_p),
            "gf2_solve_async": ([vp, vp, i64, i64, vp, i64, i64, vp], ctypes.c_int),
            "gf2_set_option": ([vp, ctypes.c_int, i64], ctypes.c_int),
            "gf2_selftest_wait": ([vp, i64], ctypes.c_int),
            "gf2_batched_config": ([vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
            "gf2_batched_get_config": ([vp, i32p], ctypes.c_int),
            "gf2_batched_autotune": ([vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
            "gf2_batched_plan_create": ([vp, ctypes.POINTER(Desc), i64, ctypes.POINTER(vp)], ctypes.c_int),
            "gf2_batched_plan_launch": ([vp, vp], ctypes.c_int),
            "gf2_batched_plan_destroy": ([vp], ctypes.c_int),
            "gf2_server_create": ([ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, i64, i64, ctypes.c_size_t],
                                  ctypes.c_int),
            "gf2_server_submit": ([vp, ctypes.POINTER(SolveJob)], ctypes.c_int),
            "gf2_server_poll": ([vp, ctypes.POINTER(SolveResult), ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
                                ctypes.c_int),
            "gf2_server_drain": ([vp], ctypes.c_int),
            "gf2_server_clock": ([], ctypes.c_double),
            "gf2_server_destroy": ([vp], ctypes.c_int),
            "gf2_carrier_check": ([ctypes.c_int, vp, vp, vp], ctypes.c_int),
            "gf2_get_timeline": ([vp, ctypes.POINTER(ctypes.c_double), i64, i64p], ctypes.c_int),
            "gf2_carrier_rate": ([ctypes.c_int, i64, ctypes.POINTER(ctypes.c_double), i64p], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
        return _lib


def strerror(code: int) -> str:
    try:
        return load().gf2_strerror(code).decode()
    except Exception:  # pragma: no cover
        return f"status {code}"


def words_for(n: int) -> int:
    return (n + 63) // 64


def _check(rc: int, what: str):
    if rc != GF2_OK:
        raise GF2Error(rc, what)


def _dptr(t) -> int:
    """Device pointer of a CUDA tensor (no copy)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return t.data_ptr()


def _mat(t, m: int, n: int):
    if t.dtype.itemsize != 8 or t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("matrix must be a 2-D tensor of 64-bit words with unit column stride")
    if t.shape[0] < m or (n > 0 and t.stride(0) < words_for(n)):
        raise ValueError("matrix too small for m x n")
    return t.stride(0)


class Handle:
    """A libgf2 handle on one CUDA device, bound to torch's current stream."""

    def __init__(self, device: int | None = None):
        import torch
        self._torch = torch
        L = load()
        dev = torch.cuda.current_device() if device is None else device
        self.device = dev
        h = ctypes.c_void_p()
        _check(L.gf2_create(ctypes.byref(h), dev), "gf2_create")
        self._h = h
        self._stream = None

    def close(self):
        if getattr(self, "_h", None):
            load().gf2_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def _bind_stream(self):
        s = self._torch.cuda.current_stream(self.device).cuda_stream
        if s != self._stream:
            _check(load().gf2_set_stream(self._h, ctypes.c_void_p(s)), "gf2_set_stream")
            self._stream = s

    # ---- decompositions ------------------------------------------------
    def ple(self, A, m: int, n: int, P, Q) -> int:
        """PLE in place; P int64[m], Q int64[min(m,n)] device tensors.  Returns the rank."""
        ld = _mat(A, m, n)
        self._bind_stream()
        rank = ctypes.c_int64(0)
        _check(load().gf2_ple(self._h, _dptr(A), m, n, ld, _dptr(P), _dptr(Q), ctypes.byref(rank)),
               "gf2_ple")
        return rank.value

    def ple_async(self, A, m: int, n: int, P, Q, rank_dev) -> None:
        ld = _mat(A, m, n)
        self._bind_stream()
        _check(load().gf2_ple_async(self._h, _dptr(A), m, n, ld, _dptr(P), _dptr(Q), _dptr(rank_dev)),
               "gf2_ple_async")

    def rref(self, A, m: int, n: int, Q) -> int:
        ld = _mat(A, m, n)
        self._bind_stream()
        rank = ctypes.c_int64(0)
        _check(load().gf2_rref(self._h, _dptr(A), m, n, ld, _dptr(Q), ctypes.byref(rank)), "gf2_rref")
        return rank.value

    def rref_async(self, A, m: int, n: int, Q, rank_dev) -> None:
        ld = _mat(A, m, n)
        self._bind_stream()
        _check(load().gf2_rref_async(self._h, _dptr(A), m, n, ld, _dptr(Q), _dptr(rank_dev)),
               "gf2_rref_async")

    def rref_m4ri(self, A, m: int, n: int, Q) -> int:
        """RREF by M4RI (Algorithm 8), in place; returns the rank."""
        ld = _mat(A, m, n)
        self._bind_stream()
        rank = ctypes.c_int64(0)
        _check(load().gf2_rref_m4ri(self._h, _dptr(A), m, n, ld, _dptr(Q), ctypes.byref(rank)), "gf2_rref_m4ri")
        return rank.value

    def rref_m4ri_async(self, A, m: int, n: int, Q, rank_dev) -> None:
        ld = _mat(A, m, n)
        self._bind_stream()
        _check(load().gf2_rref_m4ri_async(self._h, _dptr(A), m, n, ld, _dptr(Q), _dptr(rank_dev)),
               "gf2_rref_m4ri_async")

    def mul(self, C, A, B, m: int, k: int, n: int, accumulate: bool = False) -> None:
        ldc = _mat(C, m, n)
        lda = A.stride(0) if k > 0 else 1
        ldb = B.stride(0) if k > 0 else 1
        self._bind_stream()
        _check(load().gf2_mul(self._h, _dptr(C), ldc, _dptr(A) if k else None, lda,
                              _dptr(B) if k else None, ldb, m, k, n, 1 if accumulate else 0), "gf2_mul")

    def solve(self, A, B, n: int, nrhs: int) -> int:
        lda = _mat(A, n, n)
        ldb = _mat(B, n, nrhs) if nrhs > 0 else 1
        self._bind_stream()
        st = ctypes.c_int(0)
        _check(load().gf2_solve(self._h, _dptr(A), n, lda, _dptr(B) if nrhs else None, nrhs, ldb,
                                ctypes.byref(st)), "gf2_solve")
        return st.value

    def ple_batched(self, items) -> None:
        """items: sequence of (A, m, n, P, Q, rank_dev) device tensors / sizes."""
        arr = self._descs(items)
        self._bind_stream()
        _check(load().gf2_ple_batched(self._h, arr, len(items)), "gf2_ple_batched")

    @staticmethod
    def _descs(items):
        arr = (Desc * len(items))()
        for i, (A, m, n, P, Q, rk) in enumerate(items):
            ld = _mat(A, m, n)
            arr[i] = Desc(_dptr(A), m, n, ld, _dptr(P), _dptr(Q), _dptr(rk))
        return arr

    def batched_config(self, size_class: int, config: int) -> None:
        """Table configuration of the batched kernel for a size class (-1: all)."""
        _check(load().gf2_batched_config(self._h, size_class, config), "gf2_batched_config")

    def batched_get_config(self) -> list:
        out = (ctypes.c_int * BATCH_CLASSES)()
        _check(load().gf2_batched_get_config(self._h, out), "gf2_batched_get_config")
        return list(out)

    def batched_autotune(self, reps: int = 3):
        """Time every configuration per size class and keep the fastest;
        returns (chosen configs, ms[class][config])."""
        ms = (ctypes.c_double * (BATCH_CLASSES * BATCH_CONFIGS))()
        self._bind_stream()
        _check(load().gf2_batched_autotune(self._h, reps, ms), "gf2_batched_autotune")
        table = [[ms[c * BATCH_CONFIGS + k] for k in range(BATCH_CONFIGS)] for c in range(BATCH_CLASSES)]
        return self.batched_get_config(), table

    def batched_plan(self, items) -> "BatchedPlan":
        return BatchedPlan(self, items)

    def solve_async(self, A, B, n: int, nrhs: int, status_dev) -> None:
        lda = _mat(A, n, n)
        ldb = _mat(B, n, nrhs) if nrhs > 0 else 1
        self._bind_stream()
        _check(load().gf2_solve_async(self._h, _dptr(A), n, lda, _dptr(B) if nrhs else None, nrhs, ldb,
                                      _dptr(status_dev)), "gf2_solve_async")

    def workspace_bytes(self, m: int, n: int) -> int:
        return int(load().gf2_workspace_bytes(self._h, m, n))

    # ---- host-buffer forms ----------------------------------------------
    def ple_host(self, A: np.ndarray, m: int, n: int):
        """PLE of a host uint64 array in place; returns (rank, P, Q) as numpy."""
        assert A.dtype == np.uint64 and A.flags["C_CONTIGUOUS"]
        P = np.zeros(max(m, 1), dtype=np.int64)
        Q = np.zeros(max(min(m, n), 1), dtype=np.int64)
        rank = ctypes.c_int64(0)
        self._bind_stream()
        _check(load().gf2_ple_host(self._h, A.ctypes.data, m, n, A.shape[1], P.ctypes.data,
                                   Q.ctypes.data, ctypes.byref(rank)), "gf2_ple_host")
        return rank.value, P[:m], Q[:min(m, n)]

    def rref_host(self, A, m: int, n: int, Q=None) -> int:
        """RREF of a host buffer in place.  A: numpy uint64 array or a pinned
        CPU torch tensor of 64-bit words; Q likewise (int64[min(m, n)])."""
        if isinstance(A, np.ndarray):
            aptr, ld = A.ctypes.data, A.shape[1]
        else:
            aptr, ld = A.data_ptr(), A.stride(0)
        if Q is None:
            Q = np.zeros(max(min(m, n), 1), dtype=np.int64)
        qptr = Q.ctypes.data if isinstance(Q, np.ndarray) else Q.data_ptr()
        rank = ctypes.c_int64(0)
        self._bind_stream()
        _check(load().gf2_rref_host(self._h, aptr, m, n, ld, qptr, ctypes.byref(rank)), "gf2_rref_host")
        return rank.value

    def selftest_wait(self, limit_us: int = 1000) -> int:
        """Run the bounded-wait self-test; returns the status code (GF2_ETIMEOUT expected)."""
        self._bind_stream()
        return int(load().gf2_selftest_wait(self._h, int(limit_us)))

    def set_option(self, option: int, value: int) -> None:
        """An OPT_* execution option (gf2_set_option): switches take 0 / 1, block widths a
        multiple of 64 (0 off, -1 automatic), OPT_MUL_GEMM_FORMAT 4 or 8, OPT_TRSM_LEAF 1024, 2048
        or 4096; results are identical."""
        _check(load().gf2_set_option(self._h, option, int(value)), "gf2_set_option")

    # ---- statistics -----------------------------------------------------
    def set_profiling(self, level) -> None:
        """0: off, 1 (or True): time the update, RREF back-substitution and GEMM
        launches, 2: time every kernel, 3: time every 7th update launch (only those
        count in update_ms/update_bytes) and the back-substitution, 4: time every
        kernel and keep a timeline (Handle.timeline), 5: time the GEMM launches only."""
        _check(load().gf2_set_profiling(self._h, int(level)), "gf2_set_profiling")

    def stats(self) -> dict:
        s = _Stats()
        _check(load().gf2_get_stats(self._h, ctypes.byref(s)), "gf2_get_stats")
        return {f: getattr(s, f) for f, _ in _Stats._fields_}

    def timeline(self):
        """Profiling level 4: [(kind, start_ms, end_ms), ...] of the timed launches."""
        L = load()
        cnt = ctypes.c_int64(0)
        _check(L.gf2_get_timeline(self._h, None, 0, ctypes.byref(cnt)), "gf2_get_timeline")
        buf = (ctypes.c_double * (3 * max(cnt.value, 1)))()
        _check(L.gf2_get_timeline(self._h, buf, cnt.value, ctypes.byref(cnt)), "gf2_get_timeline")
        return [(int(buf[3 * i]), buf[3 * i + 1], buf[3 * i + 2]) for i in range(cnt.value)]

    def reset_stats(self) -> None:
        _check(load().gf2_reset_stats(self._h), "gf2_reset_stats")


class BatchedPlan:
    """gf2_batched_plan_*: one batch layout captured as a CUDA graph; launch()
    replays it on the current torch stream."""

    def __init__(self, handle: Handle, items):
        self._handle = handle
        self._p = ctypes.c_void_p()
        arr = Handle._descs(items)
        _check(load().gf2_batched_plan_create(handle._h, arr, len(items), ctypes.byref(self._p)),
               "gf2_batched_plan_create")

    def launch(self) -> None:
        import torch
        st = torch.cuda.current_stream().cuda_stream
        _check(load().gf2_batched_plan_launch(self._p, ctypes.c_void_p(st)), "gf2_batched_plan_launch")

    def close(self) -> None:
        if self._p:
            load().gf2_batched_plan_destroy(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


_default = {}


def default_handle(device: int | None = None) -> Handle:
    import torch
    dev = torch.cuda.current_device() if device is None else device
    h = _default.get(dev)
    if h is None:
        h = _default[dev] = Handle(dev)
    return h


def ple_noalloc(A, m: int, n: int, P, Q) -> int:
    """gf2_ple_noalloc: PLE with all scratch in the library's fixed device
    array (m, n <= 4096), for callers that cannot allocate device memory.
    Runs on torch's current stream and returns the rank."""
    import torch
    L = load()
    f = L.gf2_ple_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]
    f.restype = ctypes.c_int
    ld = _mat(A, m, n) if m > 0 and n > 0 else max(A.stride(0), 1)
    rank = ctypes.c_int64(0)
    s = torch.cuda.current_stream().cuda_stream
    _check(f(_dptr(A), m, n, ld, _dptr(P), _dptr(Q), ctypes.byref(rank), ctypes.c_void_p(s)),
           "gf2_ple_noalloc")
    return rank.value


def carrier_check(carrier: int, a_bits, b_bits, counts) -> None:
    """gf2_carrier_check: one product of bit matrices (device int64 tensors)
    on the given tensor-core carrier; counts (device int32) receives the
    AND-population counts."""
    _check(load().gf2_carrier_check(carrier, _dptr(a_bits), _dptr(b_bits), _dptr(counts)), "gf2_carrier_check")


def carrier_rate(carrier: int, iters: int):
    """gf2_carrier_rate: (multiply-adds per second over the GPU, final count)."""
    rate = ctypes.c_double(0.0)
    cnt = ctypes.c_int64(0)
    _check(load().gf2_carrier_rate(carrier, iters, ctypes.byref(rate), ctypes.byref(cnt)), "gf2_carrier_rate")
    return rate.value, cnt.value


class Server:
    """gf2_server: continuous-batching solve server (native worker thread).

    Jobs are host buffers (numpy uint64 arrays or pinned CPU torch tensors);
    the caller keeps them alive until the job's result has been polled.
    """

    def __init__(self, slots: int = 4, max_n: int = 16384, max_nrhs: int = 64,
                 hbm_budget_bytes: int = 0, device: int | None = None):
        import torch
        L = load()
        dev = torch.cuda.current_device() if device is None else device
        s = ctypes.c_void_p()
        _check(L.gf2_server_create(ctypes.byref(s), dev, slots, max_n, max_nrhs, hbm_budget_bytes),
               "gf2_server_create")
        self._s = s

    @staticmethod
    def _host(a):
        if isinstance(a, np.ndarray):
            return a.ctypes.data, a.shape[1] if a.ndim == 2 else 1
        return a.data_ptr(), a.stride(0)

    def submit(self, job_id: int, A, n: int, B, nrhs: int, X) -> None:
        pa, lda = self._host(A)
        pb, ldb = self._host(B)
        px, ldx = self._host(X)
        j = SolveJob(job_id, pa, n, lda, pb, nrhs, ldb, px, ldx)
        _check(load().gf2_server_submit(self._s, ctypes.byref(j)), "gf2_server_submit")

    def poll(self, max_results: int = 4096):
        buf = (SolveResult * max_results)()
        cnt = ctypes.c_int(0)
        _check(load().gf2_server_poll(self._s, buf, max_results, ctypes.byref(cnt)), "gf2_server_poll")
        return [(r.id, r.status, r.error, r.t_submit, r.t_start, r.t_done) for r in buf[:cnt.value]]

    def drain(self) -> None:
        _check(load().gf2_server_drain(self._s), "gf2_server_drain")

    @staticmethod
    def clock() -> float:
        return float(load().gf2_server_clock())

    def close(self) -> None:
        if getattr(self, "_s", None):
            load().gf2_server_destroy(self._s)
            self._s = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass
