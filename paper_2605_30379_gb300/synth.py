"""Seeded synthetic semi-Markov kernels shaped like the paper's workloads.

This module builds inputs only.  It holds none of the inversion arithmetic and
is shared, unchanged, by the FP64 oracle tests and the CUDA path.  numpy only.

Sojourn laws (Appendix E and Section 5 of Kordalis & Trevezas):

* discrete Weibull, discretised like the paper's shifted discrete Gamma,
  f(k) = P(k-1 <= X < k) = exp(-((k-1)/lam)^beta) - exp(-(k/lam)^beta), k >= 1;
* shifted discrete Gamma f(k) = P(k-1 <= X < k) (Appendix E, horizon scaling);
* shifted Poisson f(k) = exp(-lam) lam^(k-1)/(k-1)!, k >= 1 (Appendix E);
* continuous Lognormal Q_ij(t) = P^emb_ij Phi((log t - mu_ij)/sigma_ij)
  (Appendix E), reduced to a discrete sequence by the endpoint mean-value
  rule of Section 4.2:  A = e0 - Qbar_h with
  Qbar_h(m) = (dQ_h(m) + dQ_h(m+1))/2, dQ_h(0) = 0, dQ_h(m) = Q_h(m) - Q_h(m-1),
  so A(0) = I - Q(h)/2.

Embedded chains: each row of P^emb has a zero diagonal and Dirichlet(alpha)
off-diagonal weights (normalised Gamma(alpha) draws).

Random draw order for one model, from ``numpy.random.default_rng(seed)``:
P^emb rows i = 0..d-1 (d-1 Gamma draws each), then the d x d shape (or sigma)
matrix row-major, then the d x d scale (or mu) matrix row-major.  Batched
workloads draw model b from ``SeedSequence(seed).spawn(n)[b]``.

Arrays are float64, shape [N][d][d], time slowest.  Generation of long
horizons is split into time chunks evaluated on a thread pool; every element
is computed by the same numpy expression, so the result does not depend on
the chunking.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
from scipy import special as _sp

__all__ = [
    "dirichlet_zero_diag", "weibull_kernel", "weibull_model", "geometric_model",
    "lognormal_model", "gamma_paper_e1", "poisson_paper_e4", "poisson_paper_e2",
    "batch_models", "identity_minus",
]

_CHUNK = 2048


def _pool_map(fn, chunks):
    workers = min(len(chunks), max(1, (os.cpu_count() or 1)))
    if workers <= 1:
        return [fn(c) for c in chunks]
    with ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(fn, chunks))


def _chunks(n):
    return [(s, min(n, s + _CHUNK)) for s in range(0, n, _CHUNK)]


def dirichlet_zero_diag(rng, d, alpha=1.0):
    """Embedded chain with P_ii = 0 and Dirichlet(alpha) off-diagonal rows."""
    if d < 2:
        raise ValueError("a zero-diagonal embedded chain needs d >= 2")
    P = np.zeros((d, d))
    for i in range(d):
        g = rng.gamma(alpha, size=d - 1)
        row = g / g.sum()
        P[i, np.arange(d) != i] = row
    return P


def identity_minus(q):
    """A = e0 - q (the sequence whose inverse is the Markov renewal sequence psi)."""
    A = -np.asarray(q, dtype=np.float64)
    d = A.shape[1]
    A[0] += np.eye(d)
    return A


def weibull_kernel(P, beta, lam, N, out=None):
    """q_ij(k) = P_ij f_ij(k) with the discrete Weibull mass f above; q(0) = 0."""
    d = P.shape[0]
    q = np.empty((N, d, d)) if out is None else out

    def work(rng_):
        s, e = rng_
        k = np.arange(s, e, dtype=np.float64)[:, None, None]
        km1 = np.maximum(k - 1.0, 0.0)
        f = np.exp(-np.power(km1 / lam, beta)) - np.exp(-np.power(k / lam, beta))
        blk = P * f
        if s == 0:
            blk[0] = 0.0
        q[s:e] = blk

    _pool_map(work, _chunks(N))
    return q


def weibull_model(d, N, seed=0, alpha=1.0, shape=(0.8, 2.0), scale=(2.0, 20.0), rng=None):
    """Discrete Weibull semi-Markov kernel with a Dirichlet(alpha) zero-diagonal chain.

    Returns (q, params) with q [N][d][d] float64, q(0) = 0."""
    rng = np.random.default_rng(seed) if rng is None else rng
    P = dirichlet_zero_diag(rng, d, alpha)
    beta = rng.uniform(shape[0], shape[1], size=(d, d))
    lam = rng.uniform(scale[0], scale[1], size=(d, d))
    q = weibull_kernel(P, beta, lam, N)
    return q, {"P": P, "beta": beta, "lam": lam}


def geometric_model(d, N, seed=0, alpha=1.0, scale=(2.0, 20.0)):
    """Markov case: discrete Weibull with beta = 1 and destination-independent
    scale lam_i, i.e. geometric sojourns with p_i = 1 - exp(-1/lam_i).

    Returns (q, params) where params has P (embedded chain) and p."""
    rng = np.random.default_rng(seed)
    P = dirichlet_zero_diag(rng, d, alpha)
    lam_i = rng.uniform(scale[0], scale[1], size=d)
    lam = np.repeat(lam_i[:, None], d, axis=1)
    beta = np.ones((d, d))
    q = weibull_kernel(P, beta, lam, N)
    p = 1.0 - np.exp(-1.0 / lam_i)
    return q, {"P": P, "p": p, "lam": lam_i}


def _lognormal_Q(P, mu, sigma, t):
    """Q(t) = P * Phi((log t - mu)/sigma) for t > 0, Q(0) = 0; t has shape [n]."""
    t = np.asarray(t, dtype=np.float64)[:, None, None]
    with np.errstate(divide="ignore"):
        z = (np.log(t) - mu) / sigma
    Q = P * _sp.ndtr(z)
    Q[t[:, 0, 0] <= 0.0] = 0.0
    return Q


def lognormal_model(d, N, seed=0, h=0.05, alpha=1.0, sigma=(1.0, 2.0), mu=(0.0, 3.0), rng=None):
    """Continuous Lognormal semi-Markov kernel reduced by the endpoint mean-value rule.

    Returns (A, params): A = e0 - Qbar_h, [N][d][d] float64, with A(0) = I - Q(h)/2.
    params holds P, mu, sigma, h and the callable Q(t) for the checks."""
    rng = np.random.default_rng(seed) if rng is None else rng
    P = dirichlet_zero_diag(rng, d, alpha)
    sig = rng.uniform(sigma[0], sigma[1], size=(d, d))
    m_u = rng.uniform(mu[0], mu[1], size=(d, d))
    A = np.empty((N, d, d))

    def work(rng_):
        s, e = rng_
        # Q_h(m) for m = s-1 .. e (clamped at 0); dQ_h(m) for m = s .. e
        lo = max(s - 1, 0)
        Qh = _lognormal_Q(P, m_u, sig, h * np.arange(lo, e + 1, dtype=np.float64))
        # dQ_h(m) = Q_h(m) - Q_h(m-1) for m >= 1, dQ_h(0) = 0
        if s == 0:
            dQ = np.concatenate([np.zeros((1, d, d)), Qh[1:] - Qh[:-1]])
        else:
            dQ = Qh[1:] - Qh[:-1]
        Qbar = 0.5 * (dQ[:-1] + dQ[1:])
        A[s:e] = -Qbar
        if s == 0:
            A[0] += np.eye(d)

    _pool_map(work, _chunks(N))
    return A, {"P": P, "mu": m_u, "sigma": sig, "h": h,
               "Q": lambda t: _lognormal_Q(P, m_u, sig, t)}


# ----------------------------------------------------------------------------
# Continuous-time inputs (raw samples only: the mean-value rule itself is
# computed by the oracle and by the library, each on its own)
# ----------------------------------------------------------------------------
def lognormal_samples(d, n, seed=0, h=0.05, alpha=1.0, sigma=(1.0, 2.0), mu=(0.0, 3.0)):
    """Samples of a Lognormal semi-Markov kernel on the grid t = m h:
    Q_h(m) = Q(mh) for m = 0 .. n (n + 1 values, [n+1][d][d]) and the
    survival matrix Hbar(mh) = diag(1 - sum_j Q_ij(mh)) for m = 0 .. n-1."""
    rng = np.random.default_rng(seed)
    P = dirichlet_zero_diag(rng, d, alpha)
    sig = rng.uniform(sigma[0], sigma[1], size=(d, d))
    m_u = rng.uniform(mu[0], mu[1], size=(d, d))
    Qs = _lognormal_Q(P, m_u, sig, h * np.arange(n + 1, dtype=np.float64))
    Hbar = np.zeros((n, d, d))
    idx = np.arange(d)
    Hbar[:, idx, idx] = 1.0 - Qs[:n].sum(axis=2)
    return Qs, Hbar


# The four-state exponential benchmark of the continuous-time example
# (Section 5, Eq. (generator)): states 0 clean, 1 acquisition, 2 infection,
# 3 fraud complete; up states U = {0, 1, 2}, down state D = {3}.
GENERATOR_4STATE = np.array([[-0.2, 0.2, 0.0, 0.0],
                             [0.01, -0.11, 0.1, 0.0],
                             [0.15, 0.3, -0.85, 0.4],
                             [0.0, 0.0, 0.5, -0.5]])


def exponential_benchmark(h, n):
    """Samples of the exponential semi-Markov kernel of Eq. (generator) on
    t = m h: exit rates a_i = -G_ii, embedded chain P_ij = G_ij / a_i
    (Eq. (embedded-continuous)), Q_ij(t) = P_ij (1 - exp(-a_i t)).
    Returns Q_h(m) for m = 0 .. n, Hbar(mh) = diag(exp(-a_i mh)) and the
    up-state survival column L_U(mh) = exp(-a_i mh) (i in U) for m = 0 .. n-1,
    with the generator, U and the initial distribution (1, 0, 0, 0)."""
    G = GENERATOR_4STATE
    a = -np.diag(G)
    P = G / a[:, None]
    np.fill_diagonal(P, 0.0)
    t = h * np.arange(n + 1, dtype=np.float64)
    surv = np.exp(-np.outer(t, a))                       # [n+1][4]
    Qs = P[None, :, :] * (1.0 - surv)[:, :, None]
    Hbar = np.zeros((n, 4, 4))
    Hbar[:, np.arange(4), np.arange(4)] = surv[:n]
    U = [0, 1, 2]
    LU = surv[:n, U][:, :, None].copy()                  # [n][3][1]
    return {"Q": Qs, "Hbar": Hbar, "LU": LU, "G": G, "U": U, "alpha": np.array([1.0, 0.0, 0.0, 0.0])}


# ----------------------------------------------------------------------------
# The paper's own small examples (parameters printed in Section 5 / Appendix E)
# ----------------------------------------------------------------------------
P_EMB_3STATE = np.array([[0.0, 1.0, 0.0], [0.2, 0.0, 0.8], [1.0, 0.0, 0.0]])
_E1_GAMMA = {(0, 1): (1.8, 4.0), (1, 0): (1.6, 5.0), (1, 2): (2.2, 4.0), (2, 0): (1.9, 3.0)}
_E4_POISSON = {(0, 1): 8.0, (1, 0): 5.0, (1, 2): 10.0, (2, 0): 7.0}


def gamma_paper_e1(N):
    """Three-state horizon-scaling kernel: P^emb of Section 5.1 with shifted
    discrete Gamma sojourns f(k) = P(k-1 <= X < k), (shape, scale) of Appendix E."""
    q = np.zeros((N, 3, 3))
    k = np.arange(1, N, dtype=np.float64)
    for (i, j), (a, th) in _E1_GAMMA.items():
        f = _sp.gammainc(a, k / th) - _sp.gammainc(a, (k - 1.0) / th)
        q[1:, i, j] = P_EMB_3STATE[i, j] * f
    return q


def _shifted_poisson(lam, N):
    k = np.arange(1, N)
    logf = -lam + (k - 1) * math.log(lam) - _sp.gammaln(k)
    return np.exp(logf)


def poisson_paper_e4(N):
    """Three-state first-entrance kernel: P^emb of Section 5.1 with shifted
    Poisson sojourns lambda_12=8, lambda_21=5, lambda_23=10, lambda_31=7."""
    q = np.zeros((N, 3, 3))
    for (i, j), lam in _E4_POISSON.items():
        q[1:, i, j] = P_EMB_3STATE[i, j] * _shifted_poisson(lam, N)
    return q


def poisson_paper_e2(s, N):
    """State-dimension experiment: uniform jumps to the other states, shifted
    Poisson with lambda_ij = 3 + ((i + j) mod 4), 1-based i, j."""
    q = np.zeros((N, s, s))
    for i in range(s):
        for j in range(s):
            if i == j:
                continue
            lam = 3.0 + ((i + 1 + j + 1) % 4)
            q[1:, i, j] = _shifted_poisson(lam, N) / (s - 1)
    return q


def _batch_shape(ss, d_range, logN_range):
    rng = np.random.default_rng(ss)
    d = int(rng.integers(d_range[0], d_range[1] + 1))
    N = int(round(2.0 ** rng.uniform(*logN_range)))
    return rng, d, N


def batch_shapes(n=256, seed=0, d_range=(3, 48), logN_range=(10.0, 16.0)):
    """The (d, N) of batch_models(n, seed) without building the models."""
    return [_batch_shape(ss, d_range, logN_range)[1:] for ss in np.random.SeedSequence(seed).spawn(n)]


def batch_models(n=256, seed=0, d_range=(3, 48), logN_range=(10.0, 16.0), h=0.05,
                 max_total_coeffs=None):
    """Mixed batch: d ~ U{d_lo..d_hi}, N = round(2^U[a,b]), even-indexed draws
    discrete Weibull, odd Lognormal mean-value.  Returns a list of dicts
    {"A": [N][d][d], "d": d, "N": N, "kind": ...}.  max_total_coeffs, if set,
    stops the list once sum N d^2 would exceed it."""
    children = np.random.SeedSequence(seed).spawn(n)
    out = []
    total = 0
    for b, ss in enumerate(children):
        rng, d, N = _batch_shape(ss, d_range, logN_range)
        if max_total_coeffs is not None and total + N * d * d > max_total_coeffs:
            break
        if b % 2 == 0:
            q, _ = weibull_model(d, N, rng=rng)
            A = identity_minus(q)
            kind = "weibull"
        else:
            A, _ = lognormal_model(d, N, h=h, rng=rng)
            kind = "lognormal"
        out.append({"A": A, "d": d, "N": N, "kind": kind})
        total += N * d * d
    return out
