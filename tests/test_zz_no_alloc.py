"""mrc_inverse_noalloc: the FP64 inverse for callers that cannot allocate
device memory (its scratch is a fixed array inside libmrc).  Called through
the C ABI and compared with mrc_inverse, the allocating entry point, on two
calls in a row with different shapes, so a leftover from the first call would
show in the second.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2605_30379_gb300 import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-11  # the FP64 parity tolerance of the other GPU tests


@pytest.fixture(scope="module")
def libs():
    from paper_2605_30379_gb300 import build, mrc
    path = build.build()
    lib = ctypes.CDLL(path)
    lib.mrc_inverse_noalloc.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]
    lib.mrc_inverse_noalloc.restype = ctypes.c_int
    return lib, mrc


def _run_noalloc(lib, A):
    N, d, _ = A.shape
    psi = torch.full_like(A, float("nan"))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.mrc_inverse_noalloc(d, N, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(psi.data_ptr()), stream)
    return st, psi


def test_noalloc_matches_allocating_inverse_twice(libs):
    lib, mrc = libs
    cases = [(16, 2048, 31), (5, 1000, 32)]
    for d, N, seed in cases:
        q, _ = synth.weibull_model(d, N, seed=seed)
        A = torch.from_numpy(synth.identity_minus(q)).cuda()
        ref = mrc.inverse(A, prec="fp64")
        st, psi = _run_noalloc(lib, A)
        assert st == 0
        torch.cuda.synchronize()
        err = (psi - ref).abs().max().item()
        assert err <= TOL64, (d, N, err)


def test_noalloc_rejects_oversized_request(libs):
    lib, _ = libs
    A = torch.zeros((1 << 15, 2, 2), dtype=torch.float64, device="cuda")
    st, _ = _run_noalloc(lib, A)
    assert st == 3  # MRC_ERR_NO_MEMORY: beyond the fixed array's limit
