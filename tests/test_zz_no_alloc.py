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


def test_noalloc_matches_oracle_and_allocating_inverse_twice(libs):
    """Two calls in a row with different shapes, each against the FP64 oracle
    and against mrc_inverse.  After one warm-up call per shape (the first call
    on a device maps the library's fixed array and kernels), the calls change
    neither the device's free memory nor torch's allocations: nothing is
    allocated."""
    import oracle
    lib, mrc = libs
    cases = [(16, 2048, 31), (5, 1000, 32)]
    data = []
    for d, N, seed in cases:
        q, _ = synth.weibull_model(d, N, seed=seed)
        A_h = synth.identity_minus(q)
        A = torch.from_numpy(A_h).cuda()
        data.append((A_h, A, mrc.inverse(A, prec="fp64"), oracle.inverse_left(A_h)))
    psis = [torch.full_like(A, float("nan")) for _, A, _, _ in data]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(A, psi):
        N, d, _ = A.shape
        return lib.mrc_inverse_noalloc(d, N, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(psi.data_ptr()), stream)

    for (_, A, _, _), psi in zip(data, psis):  # warm-up: initialisation on this device
        assert call(A, psi) == 0
    torch.cuda.synchronize()
    for (_, A, ref_dev, ref), psi in zip(data, psis):
        psi.fill_(float("nan"))
        # the device's free memory and torch's allocations around the call
        # alone (torch's own temporaries below may reserve memory in between)
        torch.cuda.synchronize()
        free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        assert call(A, psi) == 0
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_allocated() == alloc0
        got = psi.cpu().numpy()
        assert np.abs(got - ref).max() <= TOL64
        assert (psi - ref_dev).abs().max().item() <= TOL64


def test_noalloc_rejects_oversized_request(libs):
    lib, _ = libs
    A = torch.zeros((1 << 15, 2, 2), dtype=torch.float64, device="cuda")
    st, _ = _run_noalloc(lib, A)
    assert st == 3  # MRC_ERR_NO_MEMORY: beyond the fixed array's limit
