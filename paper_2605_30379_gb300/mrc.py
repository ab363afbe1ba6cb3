"""ctypes binding of libmrc (the C ABI in include/mrc.h).

Argument marshalling only: tensors are passed by data pointer and the current
torch CUDA stream is passed as the cudaStream_t.  Every step of the method
runs in libmrc's CUDA kernels; there is no Python or CPU fallback, and the
first call fails loudly if libmrc.so has not been built
(``python -c "import __graft_entry__ as g; g.build()"``).

Names follow the C ABI: ``inverse``, ``inverse_batched``, ``residual``,
``transition``, ``first_entrance``, ``occupation``, ``reward``,
``renewal_visits``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmrc.so")

MRC_FP64, MRC_MIXED = 0, 1
_PREC = {"fp64": MRC_FP64, "mixed": MRC_MIXED, MRC_FP64: MRC_FP64, MRC_MIXED: MRC_MIXED}
STATUS = {0: "ok", 1: "invalid argument", 2: "A(0) is singular", 3: "out of workspace memory",
          4: "CUDA error", 5: "refinement did not reach the target residual", 6: "device wait timed out",
          7: "unimplemented"}


class MrcError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = int(status)
        super().__init__(f"libmrc {where}: {STATUS.get(self.status, self.status)} (status {self.status})")


class _Options(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("refine_sweeps", ctypes.c_int),
                ("target_residual", ctypes.c_double), ("autotune", ctypes.c_int)]


class _Report(ctypes.Structure):
    _fields_ = [("res_left_l1", ctypes.c_double), ("res_right_l1", ctypes.c_double),
                ("res_max_abs", ctypes.c_double), ("levels", ctypes.c_int), ("sweeps", ctypes.c_int),
                ("ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_lock = threading.Lock()
_ctx = {}


def load():
    """Load libmrc.so (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libmrc.so not built at {LIB_PATH}; run __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        P, I, I64, D, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
        lib.mrc_status_string.restype = ctypes.c_char_p
        lib.mrc_version.restype = ctypes.c_char_p
        lib.mrc_create.argtypes = [ctypes.POINTER(P), I, SZ]
        lib.mrc_destroy.argtypes = [P]
        lib.mrc_sync_status.argtypes = [P, P]
        lib.mrc_inverse_workspace_bytes.argtypes = [I, I64, I]
        lib.mrc_inverse_workspace_bytes.restype = SZ
        lib.mrc_inverse.argtypes = [P, I, I64, P, P, ctypes.POINTER(_Options), P, ctypes.POINTER(_Report)]
        lib.mrc_inverse_gj.argtypes = [P, I, I64, P, P, ctypes.POINTER(_Options), P, ctypes.POINTER(_Report)]
        lib.mrc_mre_solve.argtypes = [P, I, I, I64, P, P, I, P, ctypes.POINTER(_Options), P]
        lib.mrc_inverse_host.argtypes = [P, I, I64, P, P, ctypes.POINTER(_Options), P, ctypes.POINTER(_Report)]
        lib.mrc_inverse_batched.argtypes = [P, I, P, P, P, P, ctypes.POINTER(_Options), P, ctypes.POINTER(_Report)]
        lib.mrc_residual.argtypes = [P, I, I64, P, P, I, P, P, I, P, ctypes.POINTER(_Report)]
        lib.mrc_transition.argtypes = [P, I, I64, P, P, P, I, P]
        lib.mrc_first_entrance.argtypes = [P, I, I64, P, P, I, P, P, P, P, ctypes.POINTER(_Options), P]
        lib.mrc_occupation.argtypes = [P, I, I64, P, P, P, I, P, P]
        lib.mrc_reward.argtypes = [P, I, I, I64, P, P, P, I, P]
        lib.mrc_renewal_visits.argtypes = [P, I, I64, P, P, P, I, P, P]
        lib.mrc_selftest_timeout.argtypes = [P, I, P]
        for name in ("mrc_create", "mrc_destroy", "mrc_sync_status", "mrc_inverse", "mrc_inverse_gj", "mrc_inverse_batched",
                     "mrc_residual", "mrc_transition", "mrc_first_entrance", "mrc_occupation", "mrc_reward",
                     "mrc_renewal_visits", "mrc_selftest_timeout"):
            getattr(lib, name).restype = I
        _lib = lib
        return lib


def _check(st, where):
    if st != 0:
        raise MrcError(st, where)


def context(device=None):
    """Per-device default context (created on first use)."""
    lib = load()
    dev = torch.cuda.current_device() if device is None else int(device)
    with _lock:
        if dev not in _ctx:
            h = ctypes.c_void_p()
            _check(lib.mrc_create(ctypes.byref(h), dev, 0), "mrc_create")
            _ctx[dev] = h
        return _ctx[dev]


def create_context(device=None, max_workspace_bytes=0):
    """A context of its own (mrc_create) with a workspace cap; free it with
    destroy_context."""
    lib = load()
    dev = torch.cuda.current_device() if device is None else int(device)
    h = ctypes.c_void_p()
    _check(lib.mrc_create(ctypes.byref(h), dev, int(max_workspace_bytes)), "mrc_create")
    return h


def destroy_context(h):
    _check(load().mrc_destroy(h), "mrc_destroy")


def workspace_bytes(d, N, prec="fp64"):
    """mrc_inverse_workspace_bytes."""
    return int(load().mrc_inverse_workspace_bytes(int(d), int(N), _PREC[prec]))


def release():
    """Destroy the per-device default contexts (frees their workspace and writes
    the autotuning cache when MRC_AUTOTUNE_CACHE is set); later calls create
    new ones."""
    lib = load()
    with _lock:
        for dev, h in list(_ctx.items()):
            lib.mrc_destroy(h)
            del _ctx[dev]


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _seq(x, name):
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64):
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if x.dim() != 3:
        raise ValueError(f"{name} must have shape [N, r, c]")
    return x.contiguous()


def _ptr(x):
    return ctypes.c_void_p(x.data_ptr()) if x is not None else ctypes.c_void_p(0)


def _opts(prec, sweeps, target, autotune=False):
    return _Options(_PREC[prec], int(sweeps), float(target), 1 if autotune else 0)


def inverse(A, prec="fp64", sweeps=1, target_residual=0.0, report=False, out=None, stream=None, autotune=False):
    """psi = A^{(-1)} mod x^N (mrc_inverse).  A: CUDA float64 [N, d, d]."""
    A = _seq(A, "A")
    N, d, d2 = A.shape
    if d != d2:
        raise ValueError("A must be square per coefficient")
    psi = torch.empty_like(A) if out is None else out
    rep = _Report()
    st = load().mrc_inverse(context(A.device.index), d, N, _ptr(A), _ptr(psi),
                            ctypes.byref(_opts(prec, sweeps, target_residual, autotune)), _stream(stream),
                            ctypes.byref(rep) if report else None)
    _check(st, "mrc_inverse")
    return (psi, rep.as_dict()) if report else psi


def inverse_gj(A, report=False, out=None, stream=None, autotune=False):
    """psi = A^{(-1)} mod x^N by series Gauss-Jordan elimination
    (mrc_inverse_gj, FP64).  A: CUDA float64 [N, d, d], d <= 64."""
    A = _seq(A, "A")
    N, d, d2 = A.shape
    if d != d2:
        raise ValueError("A must be square per coefficient")
    psi = torch.empty_like(A) if out is None else out
    rep = _Report()
    st = load().mrc_inverse_gj(context(A.device.index), d, N, _ptr(A), _ptr(psi),
                               ctypes.byref(_opts("fp64", 0, 0.0, autotune)), _stream(stream),
                               ctypes.byref(rep) if report else None)
    _check(st, "mrc_inverse_gj")
    return (psi, rep.as_dict()) if report else psi


def inverse_host(A, prec="fp64", sweeps=1, target_residual=0.0, report=False, out=None, stream=None,
                 autotune=False, device=None):
    """psi = A^{(-1)} mod x^N from host memory (mrc_inverse_host): A is a CPU
    float64 tensor [N, d, d] (pinned memory lets the upload overlap the
    Newton levels); the result is written into `out` (a CPU tensor, pinned
    preferred), valid once the stream has been synchronised (a report
    synchronises)."""
    if not (isinstance(A, torch.Tensor) and not A.is_cuda and A.dtype == torch.float64 and A.dim() == 3):
        raise TypeError("A must be a CPU float64 tensor [N, d, d]")
    A = A.contiguous()
    N, d, d2 = A.shape
    if d != d2:
        raise ValueError("A must be square per coefficient")
    psi = torch.empty_like(A) if out is None else out
    if psi.is_cuda or psi.dtype != torch.float64 or psi.shape != A.shape or not psi.is_contiguous():
        raise TypeError("out must be a contiguous CPU float64 tensor shaped like A")
    rep = _Report()
    st = load().mrc_inverse_host(context(device), d, N, _ptr(A), _ptr(psi),
                                 ctypes.byref(_opts(prec, sweeps, target_residual, autotune)), _stream(stream),
                                 ctypes.byref(rep) if report else None)
    _check(st, "mrc_inverse_host")
    return (psi, rep.as_dict()) if report else psi


def mre_solve(Q, L, scheme="mean_value", prec="fp64", sweeps=1, stream=None):
    """K_h for the continuous-time equation K = L + Q * K (mrc_mre_solve).
    Q: CUDA float64 [N+1, d, d] kernel samples Q(mh), m = 0..N; L: [N, d, c];
    scheme "mean_value" (Eq. (mre-solution)) or "process" (Eq.
    (process-discretization))."""
    Q, L = _seq(Q, "Q"), _seq(L, "L")
    N, d, c = L.shape
    if Q.shape != (N + 1, d, d):
        raise ValueError("Q must be [N+1, d, d] for L of shape [N, d, c]")
    K = torch.empty_like(L)
    sc = {"mean_value": 0, "process": 1}[scheme]
    _check(load().mrc_mre_solve(context(L.device.index), d, c, N, _ptr(Q), _ptr(L), sc, _ptr(K),
                                ctypes.byref(_opts(prec, sweeps, 0.0)), _stream(stream)), "mrc_mre_solve")
    return K


def inverse_batched(As, prec="fp64", sweeps=1, outs=None, report=False, stream=None, autotune=False, ctx=None):
    """mrc_inverse_batched over a list of independent models (ctx: a context
    from create_context, else the device's default one)."""
    As = [_seq(a, "A") for a in As]
    outs = [torch.empty_like(a) for a in As] if outs is None else outs
    n = len(As)
    dv = (ctypes.c_int * n)(*[a.shape[1] for a in As])
    Nv = (ctypes.c_int64 * n)(*[a.shape[0] for a in As])
    Ap = (ctypes.c_void_p * n)(*[a.data_ptr() for a in As])
    Pp = (ctypes.c_void_p * n)(*[p.data_ptr() for p in outs])
    reps = (_Report * n)() if report else None
    dev = As[0].device.index if n else None
    st = load().mrc_inverse_batched(context(dev) if ctx is None else ctx, n, dv, Nv, Ap, Pp,
                                    ctypes.byref(_opts(prec, sweeps, 0.0, autotune)), _stream(stream), reps)
    _check(st, "mrc_inverse_batched")
    return (outs, [r.as_dict() for r in reps]) if report else outs


def residual(A, psi, sides=3, prec="fp64", want_rho=True, stream=None):
    """(rho_L, rho_R, report) with rho_L = e0 - A*psi, rho_R = e0 - psi*A (mrc_residual).
    The report always synchronises; rho tensors are None when not asked for."""
    A, psi = _seq(A, "A"), _seq(psi, "psi")
    N, d, _ = A.shape
    rl = torch.empty_like(A) if (want_rho and sides & 1) else None
    rr = torch.empty_like(A) if (want_rho and sides & 2) else None
    rep = _Report()
    st = load().mrc_residual(context(A.device.index), d, N, _ptr(A), _ptr(psi), int(sides), _ptr(rl), _ptr(rr),
                             _PREC[prec], _stream(stream), ctypes.byref(rep))
    _check(st, "mrc_residual")
    return rl, rr, rep.as_dict()


def transition(psi, q, prec="fp64", stream=None):
    """P = psi * Hbar (mrc_transition)."""
    psi, q = _seq(psi, "psi"), _seq(q, "q")
    N, d, _ = psi.shape
    P = torch.empty_like(psi)
    _check(load().mrc_transition(context(psi.device.index), d, N, _ptr(psi), _ptr(q), _ptr(P), _PREC[prec],
                                 _stream(stream)), "mrc_transition")
    return P


def first_entrance(q, D, alpha_C, prec="fp64", sweeps=1, stream=None):
    """(g_D, F_D, S_D) for target set D (mrc_first_entrance)."""
    q = _seq(q, "q")
    N, d, _ = q.shape
    D = [int(x) for x in D]
    nC, nD = d - len(D), len(D)
    alpha_C = alpha_C.to(device=q.device, dtype=torch.float64).contiguous()
    g = torch.empty((N, nC, nD), dtype=torch.float64, device=q.device)
    F = torch.empty(N, dtype=torch.float64, device=q.device)
    S = torch.empty(N, dtype=torch.float64, device=q.device)
    Dv = (ctypes.c_int * nD)(*D)
    st = load().mrc_first_entrance(context(q.device.index), d, N, _ptr(q), Dv, nD, _ptr(alpha_C), _ptr(g), _ptr(F),
                                   _ptr(S), ctypes.byref(_opts(prec, sweeps, 0.0)), _stream(stream))
    _check(st, "mrc_first_entrance")
    return g, F, S


def occupation(P, alpha, B, stream=None):
    """A_B(k) = alpha P(k) 1_B (mrc_occupation); availability with B = up states."""
    P = _seq(P, "P")
    N, d, _ = P.shape
    alpha = alpha.to(device=P.device, dtype=torch.float64).contiguous()
    out = torch.empty(N, dtype=torch.float64, device=P.device)
    B = [int(x) for x in B]
    Bv = (ctypes.c_int * max(1, len(B)))(*B)
    _check(load().mrc_occupation(context(P.device.index), d, N, _ptr(P), _ptr(alpha), Bv, len(B), _ptr(out),
                                 _stream(stream)), "mrc_occupation")
    return out


def reward(psi, r, prec="fp64", stream=None):
    """V = psi * r (mrc_reward); r: CUDA float64 [N, d, c]."""
    psi, r = _seq(psi, "psi"), _seq(r, "r")
    N, d, _ = psi.shape
    if r.shape[0] != N or r.shape[1] != d:
        raise ValueError("r must have shape [N, d, c]")
    V = torch.empty_like(r)
    _check(load().mrc_reward(context(psi.device.index), d, r.shape[2], N, _ptr(psi), _ptr(r), _ptr(V), _PREC[prec],
                             _stream(stream)), "mrc_reward")
    return V


def renewal_visits(psi, alpha, B, stream=None):
    """N_B(k) = alpha sum_{l<=k} psi(l) I_B 1 (mrc_renewal_visits)."""
    psi = _seq(psi, "psi")
    N, d, _ = psi.shape
    alpha = alpha.to(device=psi.device, dtype=torch.float64).contiguous()
    out = torch.empty(N, dtype=torch.float64, device=psi.device)
    B = [int(x) for x in B]
    Bv = (ctypes.c_int * max(1, len(B)))(*B)
    _check(load().mrc_renewal_visits(context(psi.device.index), d, N, _ptr(psi), _ptr(alpha), Bv, len(B), _ptr(out),
                                     _stream(stream)), "mrc_renewal_visits")
    return out


def selftest_timeout(spins=256, stream=None):
    """Enqueue the bounded-wait self-test (mrc_selftest_timeout): a device
    wait on a barrier nothing arrives on gives up after `spins` rounds and
    leaves MRC_ERR_TIMEOUT in the context's status word."""
    _check(load().mrc_selftest_timeout(context(), int(spins), _stream(stream)), "mrc_selftest_timeout")


def sync_status(stream=None):
    _check(load().mrc_sync_status(context(), _stream(stream)), "mrc_sync_status")


def workspace_bytes(d, N, prec="fp64"):
    return int(load().mrc_inverse_workspace_bytes(int(d), int(N), _PREC[prec]))
