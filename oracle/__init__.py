"""FP64 CPU oracle for matrix renewal convolution (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
product path never imports or calls it, and the two share no code: the oracle
is plain C (``mrc_oracle.c``) compiled with gcc, loaded here through ctypes.

Every function follows a definition in Kordalis & Trevezas (arXiv 2605.30379):

* ``inverse_left``   -- A(0) psi(k) = delta(k) I - sum_{l=1..k} A(l) psi(k-l)
                        (Theorem 2.2; Eq. (renewal-sequence) when A = e0 - q)
* ``inverse_right``  -- Eq. (inverse-recursion)
* ``convolve``       -- Eq. (convolution)
* ``residuals``      -- rho_L, rho_R of Proposition 2.6 (and one entry at one
                        time index: ``residual_left_entry`` / ``_right_entry``)
* ``transition``     -- P = psi * Hbar, Eq. (transition-discrete)
* ``first_entrance`` -- Eqs. (first-entrance-mass), (first-entrance-cdf)
* ``occupation``     -- A_B(k) = alpha P(k) 1_{E,B} (Table 2; availability)
* ``renewal_visits`` -- Eq. (renewal-visits)
* ``mean_value_terms`` / ``mre_solve`` -- the endpoint mean-value rule and
                        Eq. (mre-solution) for K = L + Q * K in continuous time
* ``process_discretization`` -- Eq. (process-discretization)
* ``norm1_frob`` / ``norm1_spec`` -- the horizon norm ||.||_{1,N} of Section 2

Parity pins for each of these live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mrc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libmrc_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FP contraction) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i64, c_int, c_dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            p = ctypes.c_void_p
            lib.orc_gauss_jordan.argtypes = [c_int, p, p]
            lib.orc_convolve.argtypes = [c_int, c_int, c_int, i64, p, p, p]
            lib.orc_inverse_left.argtypes = [c_int, i64, p, p]
            lib.orc_inverse_right.argtypes = [c_int, i64, p, p]
            lib.orc_residuals.argtypes = [c_int, i64, p, p, p, p]
            lib.orc_residual_left_at.argtypes = [c_int, i64, p, p, p]
            lib.orc_residual_left_entry.argtypes = [c_int, i64, c_int, c_int, p, p]
            lib.orc_residual_left_entry.restype = c_dbl
            lib.orc_residual_right_entry.argtypes = [c_int, i64, c_int, c_int, p, p]
            lib.orc_residual_right_entry.restype = c_dbl
            lib.orc_hbar.argtypes = [c_int, i64, p, p]
            lib.orc_transition.argtypes = [c_int, i64, p, p, p]
            lib.orc_first_entrance.argtypes = [c_int, i64, p, p, p, p, p, p]
            lib.orc_occupation.argtypes = [c_int, i64, p, p, p, p]
            lib.orc_renewal_visits.argtypes = [c_int, i64, p, p, p, p]
            lib.orc_norm1_frob.argtypes = [c_int, c_int, i64, p]
            lib.orc_norm1_frob.restype = c_dbl
            lib.orc_norm1_spec.argtypes = [c_int, c_int, i64, p]
            lib.orc_norm1_spec.restype = c_dbl
            lib.orc_spectral_norm.argtypes = [c_int, c_int, p]
            lib.orc_spectral_norm.restype = c_dbl
            lib.orc_num_threads.restype = c_int
            _lib = lib
    return _lib


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class SingularA0(ValueError):
    """A(0) is singular, so the sequence has no convolutional inverse (Theorem 2.2)."""


def num_threads() -> int:
    return int(_load().orc_num_threads())


def gauss_jordan(M):
    M = _f64(M)
    d = M.shape[0]
    out = np.empty_like(M)
    if _load().orc_gauss_jordan(d, _ptr(M), _ptr(out)):
        raise SingularA0("singular matrix")
    return out


def convolve(A, B, N=None):
    """C(k) = sum_{l<=k} A(l) B(k-l) for k < N (Eq. (convolution))."""
    A, B = _f64(A), _f64(B)
    N = A.shape[0] if N is None else N
    assert A.shape[0] >= N and B.shape[0] >= N
    r, m = A.shape[1], A.shape[2]
    m2, c = B.shape[1], B.shape[2]
    assert m == m2
    C = np.empty((N, r, c))
    _load().orc_convolve(r, m, c, N, _ptr(A), _ptr(B), _ptr(C))
    return C


def inverse_left(A):
    A = _f64(A)
    N, d, _ = A.shape
    psi = np.empty_like(A)
    if _load().orc_inverse_left(d, N, _ptr(A), _ptr(psi)):
        raise SingularA0("A(0) is singular")
    return psi


def inverse_right(A):
    A = _f64(A)
    N, d, _ = A.shape
    psi = np.empty_like(A)
    if _load().orc_inverse_right(d, N, _ptr(A), _ptr(psi)):
        raise SingularA0("A(0) is singular")
    return psi


inverse = inverse_left


def residuals(A, psi):
    """(rho_L, rho_R) = (e0 - A*psi, e0 - psi*A) over the horizon (Proposition 2.6)."""
    A, psi = _f64(A), _f64(psi)
    N, d, _ = A.shape
    rl, rr = np.empty_like(A), np.empty_like(A)
    _load().orc_residuals(d, N, _ptr(A), _ptr(psi), _ptr(rl), _ptr(rr))
    return rl, rr


def residual_left_at(A, psi, k):
    """rho_L(k) for one time index k (cost O(k d^3))."""
    A, psi = _f64(A[: k + 1]), _f64(psi[: k + 1])
    d = A.shape[1]
    out = np.empty((d, d))
    _load().orc_residual_left_at(d, k, _ptr(A), _ptr(psi), _ptr(out))
    return out


def _prefix_view(X, k):
    """X[: k + 1] as a C-contiguous float64 array, without copying when X
    already is one (the sampled residuals of very long runs)."""
    X = X[: k + 1]
    if X.dtype == np.float64 and X.flags["C_CONTIGUOUS"]:
        return X
    return _f64(X)


def residual_left_entry(A, psi, k, i, j):
    """rho_L(k)_{ij} = delta(k) delta_{ij} - sum_{l<=k} (A(l) psi(k-l))_{ij}
    (Proposition 2.6) for one entry and one time index (cost O(k d))."""
    A, psi = _prefix_view(A, k), _prefix_view(psi, k)
    d = A.shape[1]
    return float(_load().orc_residual_left_entry(d, k, i, j, _ptr(A), _ptr(psi)))


def residual_right_entry(A, psi, k, i, j):
    """rho_R(k)_{ij} = delta(k) delta_{ij} - sum_{l<=k} (psi(l) A(k-l))_{ij}."""
    A, psi = _prefix_view(A, k), _prefix_view(psi, k)
    d = A.shape[1]
    return float(_load().orc_residual_right_entry(d, k, i, j, _ptr(A), _ptr(psi)))


def hbar(q):
    q = _f64(q)
    N, d, _ = q.shape
    out = np.empty((N, d))
    _load().orc_hbar(d, N, _ptr(q), _ptr(out))
    return out


def transition(psi, q):
    psi, q = _f64(psi), _f64(q)
    N, d, _ = psi.shape
    P = np.empty_like(psi)
    _load().orc_transition(d, N, _ptr(psi), _ptr(q), _ptr(P))
    return P


def first_entrance(q, D, alphaC):
    """Returns (g_D [N][|C|][|D|], F_D [N], S_D [N]) for target set D (list of state indices)."""
    q = _f64(q)
    N, d, _ = q.shape
    inD = np.zeros(d, dtype=np.int32)
    inD[list(D)] = 1
    nC, nD = d - int(inD.sum()), int(inD.sum())
    alphaC = _f64(alphaC)
    assert alphaC.shape == (nC,)
    g = np.empty((N, nC, nD))
    F = np.empty(N)
    S = np.empty(N)
    rc = _load().orc_first_entrance(d, N, _ptr(q), _ptr(inD), _ptr(alphaC), _ptr(g), _ptr(F), _ptr(S))
    if rc == 1:
        raise SingularA0("e0^C - q_CC is not invertible")
    if rc:
        raise ValueError("C and D must both be non-empty")
    return g, F, S


def occupation(P, alpha, B):
    P, alpha = _f64(P), _f64(alpha)
    N, d, _ = P.shape
    inB = np.zeros(d, dtype=np.int32)
    inB[list(B)] = 1
    out = np.empty(N)
    _load().orc_occupation(d, N, _ptr(P), _ptr(alpha), _ptr(inB), _ptr(out))
    return out


def renewal_visits(psi, alpha, B):
    psi, alpha = _f64(psi), _f64(alpha)
    N, d, _ = psi.shape
    inB = np.zeros(d, dtype=np.int32)
    inB[list(B)] = 1
    out = np.empty(N)
    _load().orc_renewal_visits(d, N, _ptr(psi), _ptr(alpha), _ptr(inB), _ptr(out))
    return out


def norm1_frob(X):
    X = _f64(X)
    N, r, c = X.shape
    return float(_load().orc_norm1_frob(r, c, N, _ptr(X)))


def norm1_spec(X):
    X = _f64(X)
    N, r, c = X.shape
    return float(_load().orc_norm1_spec(r, c, N, _ptr(X)))


def spectral_norm(M):
    M = _f64(M)
    r, c = M.shape
    return float(_load().orc_spectral_norm(r, c, _ptr(M)))


def mean_value_terms(Qs):
    """The endpoint mean-value rule of Section 4: from the kernel samples
    Q_h(m) = Q(mh), m = 0 .. n (the extra value Q_h(n) serves Delta+ at
    n - 1), the increments Delta Q_h(0) = O, Delta Q_h(m) = Q_h(m) - Q_h(m-1),
    Delta+ Q_h(m) = Delta Q_h(m+1) and Qbar_h(m) = (Delta Q_h(m) +
    Delta+ Q_h(m)) / 2 for m = 0 .. n-1.  Returns (dQ, dQplus, Qbar)."""
    Qs = _f64(Qs)
    n = Qs.shape[0] - 1
    dQ = np.zeros((n + 1,) + Qs.shape[1:])
    dQ[1:] = Qs[1:] - Qs[:-1]
    dQplus = dQ[1:n + 1]
    Qbar = 0.5 * (dQ[:n] + dQplus)
    return dQ[:n], dQplus, Qbar


def mre_solve(Qs, L):
    """Eq. (mre-solution): K_h = (e0 - Qbar_h)^(-1) * [L_h - (1/2) Delta+ Q_h *
    (L_h(0) e0)], the mean-value discretisation Eq. (mre-discrete) of
    K = L + Q * K.  Qs: Q_h(m), m = 0 .. n; L: [n][d][c].  The term
    Delta+ Q_h * (L_h(0) e0) is Delta+ Q_h(k) L_h(0) at every k."""
    _, dQplus, Qbar = mean_value_terms(Qs)
    L = _f64(L)
    n, d = L.shape[0], L.shape[1]
    A = -Qbar
    A[0] += np.eye(d)
    psi = inverse_left(A)
    R = L - 0.5 * np.einsum("kij,jc->kic", dQplus, L[0])
    return convolve(psi, R)


def process_discretization(Qs, L):
    """Eq. (process-discretization) with a general right-hand side:
    (e0 - Delta Q_h)^(-1) * L_h (L = Hbar_h gives the transition function)."""
    dQ, _, _ = mean_value_terms(Qs)
    L = _f64(L)
    d = L.shape[1]
    A = -dQ
    A[0] += np.eye(d)
    return convolve(inverse_left(A), L)
