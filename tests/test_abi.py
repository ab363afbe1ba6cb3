"""The C-ABI library loads and exports every entry point include/mrc.h declares
(no device calls: these run on a machine without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mrc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mrc_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_30379_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for n in ("mrc_inverse", "mrc_transition", "mrc_first_entrance", "mrc_residual", "mrc_inverse_batched"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_argument_errors(lib):
    lib.mrc_inverse.restype = ctypes.c_int
    lib.mrc_inverse.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.mrc_inverse(None, 4, 16, None, None, None, None, None) == 1  # MRC_ERR_INVALID_ARG
    lib.mrc_status_string.restype = ctypes.c_char_p
    assert lib.mrc_status_string(2) == b"A(0) is singular"
    lib.mrc_inverse_workspace_bytes.restype = ctypes.c_size_t
    lib.mrc_inverse_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int]
    assert lib.mrc_inverse_workspace_bytes(0, 16, 0) == 0
    small = lib.mrc_inverse_workspace_bytes(4, 1024, 0)
    big = lib.mrc_inverse_workspace_bytes(64, 1 << 18, 1)
    assert 0 < small < big


def test_product_path_has_no_oracle_or_cpu_fallback():
    """The binding and the CUDA sources never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_2605_30379_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
