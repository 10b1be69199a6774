"""The C ABI library builds for sm_103a, loads, and exports every declared symbol.

No GPU is needed: only symbol lookup, the status strings and argument
validation that fails before any CUDA call are exercised.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gf2.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(gf2_[a-z_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1111_6549_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["gf2_create", "gf2_destroy", "gf2_set_stream", "gf2_ple", "gf2_rref", "gf2_mul",
                 "gf2_solve", "gf2_ple_batched", "gf2_workspace_bytes", "gf2_strerror"]:
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_validation_without_gpu(lib):
    lib.gf2_strerror.restype = ctypes.c_char_p
    assert lib.gf2_strerror(0) == b"GF2_OK"
    assert b"invalid" in lib.gf2_strerror(1)
    assert b"unknown" in lib.gf2_strerror(99)
    # null handle / null output pointers are rejected before any CUDA call
    lib.gf2_ple.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                            ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.gf2_ple(None, None, 4, 4, 1, None, None, None) == 1
    lib.gf2_create.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.gf2_create(None, 0) == 1
    lib.gf2_mul.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p, ctypes.c_int64] * 3 + \
        [ctypes.c_int64] * 3 + [ctypes.c_int]
    assert lib.gf2_mul(None, None, 1, None, 1, None, 1, 4, 4, 4, 0) == 1


def test_library_built_for_sm103a():
    from paper_1111_6549_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.exists(build.LIB)


def test_binding_constants_match_the_header():
    """Every status, solve-status and option number the Python binding uses is
    the one include/gf2.h defines (the binding marshals plain integers)."""
    import paper_1111_6549_gb300 as g
    defines = dict((k, int(v)) for k, v in
                   re.findall(r"^#define\s+(GF2_[A-Z0-9_]+)\s+(-?\d+)", open(HEADER).read(), flags=re.M))
    checked = 0
    for name, value in defines.items():
        py = name if name.startswith(("GF2_OK", "GF2_E")) else name[len("GF2_"):]
        if hasattr(g, py):
            assert getattr(g, py) == value, (name, getattr(g, py), value)
            checked += 1
    opts = [k for k in defines if k.startswith("GF2_OPT_")]
    assert opts and all(hasattr(g, k[len("GF2_"):]) for k in opts)
    assert checked >= len(opts) + 6 + 3
