"""Helpers shared by the GPU parity tests: host <-> device copies of packed matrices."""
import numpy as np


def to_dev(A: np.ndarray, ld: int | None = None):
    """numpy uint64 (m, w) -> CUDA int64 tensor (m, ld) holding the same words."""
    import torch
    m, w = A.shape
    ld = w if ld is None else ld
    out = np.zeros((m, max(ld, 1)), dtype=np.uint64)
    out[:, :w] = A
    return torch.from_numpy(out.view(np.int64)).cuda()


def to_host(t, w: int | None = None) -> np.ndarray:
    a = t.cpu().numpy().view(np.uint64)
    return np.ascontiguousarray(a if w is None else a[:, :w])


def vec_dev(n: int, fill: int = -7):
    import torch
    return torch.full((max(n, 1),), fill, dtype=torch.int64, device="cuda")


def library_gemm_available() -> bool:
    """True when libgf2 was built with the library-GEMM form of the product
    (GF2_WITH_CUBLASLT=1); the default build has only its own kernels."""
    import paper_1111_6549_gb300 as g
    h = g.Handle()
    try:
        h.set_option(g.OPT_MUL_GEMM_FORMAT, 4)
        return True
    except g.GF2Error:
        return False
    finally:
        h.close()
