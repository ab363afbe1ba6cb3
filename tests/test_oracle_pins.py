"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's own formula: each compares it with an
exact rational computation, a closed form derived by hand, a library routine
(numpy), an invariant the paper proves, or a number the paper prints.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2605_30379_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers
def _rand_rational_seq(rng, N, d, a0=None, denom=7):
    """Exact rational sequence; A(0) given or zero."""
    seq = []
    for k in range(N):
        if k == 0 and a0 is not None:
            seq.append([[Fraction(x) for x in row] for row in a0])
            continue
        if k == 0:
            seq.append([[Fraction(0)] * d for _ in range(d)])
            continue
        seq.append([[Fraction(int(rng.integers(0, denom)), denom * d) for _ in range(d)] for _ in range(d)])
    return seq


def _mm(X, Y):
    return [[sum((X[i][t] * Y[t][j] for t in range(len(Y))), Fraction(0)) for j in range(len(Y[0]))]
            for i in range(len(X))]


def _madd(X, Y):
    return [[X[i][j] + Y[i][j] for j in range(len(X[0]))] for i in range(len(X))]


def _zero(d):
    return [[Fraction(0)] * d for _ in range(d)]


def _eye(d):
    return [[Fraction(int(i == j)) for j in range(d)] for i in range(d)]


def _conv_exact(A, B):
    N, d = len(A), len(A[0])
    out = []
    for k in range(N):
        s = _zero(d)
        for l in range(k + 1):
            s = _madd(s, _mm(A[l], B[k - l]))
        out.append(s)
    return out


def _inv_adjugate(M):
    """Exact inverse of a 2x2 or 3x3 rational matrix by cofactors / determinant."""
    d = len(M)
    if d == 1:
        return [[1 / M[0][0]]]
    if d == 2:
        det = M[0][0] * M[1][1] - M[0][1] * M[1][0]
        return [[M[1][1] / det, -M[0][1] / det], [-M[1][0] / det, M[0][0] / det]]
    assert d == 3
    (a, b, c), (e, f, g), (h, i, j) = M
    det = a * (f * j - g * i) - b * (e * j - g * h) + c * (e * i - f * h)
    cof = [[f * j - g * i, -(e * j - g * h), e * i - f * h],
           [-(b * j - c * i), a * j - c * h, -(a * i - b * h)],
           [b * g - c * f, -(a * g - c * e), a * f - b * e]]
    return [[cof[jj][ii] / det for jj in range(3)] for ii in range(3)]


def _to_np(seq):
    return np.array([[[float(x) for x in row] for row in m] for m in seq])


# ------------------------------------------------------- Theorem 2.2 pins
@pytest.mark.parametrize("d,N,seed", [(1, 9, 0), (2, 8, 1), (3, 7, 2)])
def test_neumann_series_exact(d, N, seed):
    """psi = sum_n q^(n) (Eq. (renewal-sequence)) in exact rationals."""
    rng = np.random.default_rng(seed)
    q = _rand_rational_seq(rng, N, d)
    e0 = [_eye(d)] + [_zero(d) for _ in range(N - 1)]
    psi = [_zero(d) for _ in range(N)]
    power = e0
    for _ in range(N):  # q^(n)(k) = 0 for n > k, so N terms are exact on the horizon
        psi = [_madd(psi[k], power[k]) for k in range(N)]
        power = _conv_exact(q, power)
    A = synth.identity_minus(_to_np(q))
    ref = _to_np(psi)
    for got in (oracle.inverse_left(A), oracle.inverse_right(A)):
        np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("d,N,seed", [(2, 7, 3), (3, 6, 4)])
def test_theorem_2_2_general_A0(d, N, seed):
    """A^(-1) = D * sum_n (e0 - A*D)^(n), D(0) = A(0)^{-1}, exact rationals."""
    rng = np.random.default_rng(seed)
    a0 = [[Fraction(int(rng.integers(1, 9)), 5) + (Fraction(2) if i == j else 0) for j in range(d)]
          for i in range(d)]
    A = _rand_rational_seq(rng, N, d, a0=a0)
    A = [[[-x for x in row] for row in m] if k else m for k, m in enumerate(A)]  # mixed signs
    Dinv = _inv_adjugate(A[0])
    D = [Dinv] + [_zero(d) for _ in range(N - 1)]
    At = _conv_exact(A, D)
    e0 = [_eye(d)] + [_zero(d) for _ in range(N - 1)]
    C = [[[e0[k][i][j] - At[k][i][j] for j in range(d)] for i in range(d)] for k in range(N)]
    S = [_zero(d) for _ in range(N)]
    power = e0
    for _ in range(N):
        S = [_madd(S[k], power[k]) for k in range(N)]
        power = _conv_exact(C, power)
    ref = _to_np(_conv_exact(D, S))
    An = _to_np(A)
    np.testing.assert_allclose(oracle.inverse_left(An), ref, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(oracle.inverse_right(An), ref, rtol=1e-12, atol=1e-14)


def test_singular_A0_detected():
    A = np.zeros((4, 2, 2))
    A[0] = [[1.0, 2.0], [2.0, 4.0]]
    with pytest.raises(oracle.SingularA0):
        oracle.inverse_left(A)
    with pytest.raises(oracle.SingularA0):
        oracle.inverse_right(A)


def test_gauss_jordan_vs_numpy():
    rng = np.random.default_rng(5)
    for d in (1, 2, 5, 17, 40):
        M = rng.standard_normal((d, d)) + d * np.eye(d)
        np.testing.assert_allclose(oracle.gauss_jordan(M), np.linalg.inv(M), rtol=1e-12, atol=1e-13)
    # a row permutation is needed: zero leading pivot
    M = np.array([[0.0, 1.0, 2.0], [3.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
    np.testing.assert_allclose(oracle.gauss_jordan(M) @ M, np.eye(3), atol=1e-14)


# --------------------------------------------------------- closed forms
def test_scalar_two_step_closed_form():
    """q(1) = q(2) = 1/2:  psi = 1/((1-x)(1+x/2)) => psi(k) = 2/3 + (1/3)(-1/2)^k."""
    N = 400
    q = np.zeros((N, 1, 1))
    q[1] = q[2] = 0.5
    psi = oracle.inverse_left(synth.identity_minus(q))[:, 0, 0]
    k = np.arange(N)
    np.testing.assert_allclose(psi, 2 / 3 + (1 / 3) * (-0.5) ** k, rtol=0, atol=1e-15)
    assert [Fraction(x).limit_denominator(64) for x in psi[:5]] == [1, Fraction(1, 2), Fraction(3, 4),
                                                                    Fraction(5, 8), Fraction(11, 16)]


def test_scalar_geometric_and_general_A0():
    """q(k) = (1-p)^{k-1} p gives psi(k) = p for k >= 1; A(k) = a r^k gives
    A^(-1) = (1 - r x)/a, i.e. (1/a, -r/a, 0, 0, ...)."""
    N, p = 300, 0.3
    k = np.arange(N)
    q = np.where(k >= 1, (1 - p) ** np.maximum(k - 1, 0) * p, 0.0)[:, None, None]
    psi = oracle.inverse_left(synth.identity_minus(q))[:, 0, 0]
    assert psi[0] == 1.0
    # the recursion sums k terms: its rounding error is at most a few k u
    assert np.all(np.abs(psi[1:] - p) <= 4 * k[1:] * 2.0 ** -53)
    a, r = 2.5, 0.7
    A = (a * r ** k)[:, None, None]
    for inv in (oracle.inverse_left(A), oracle.inverse_right(A)):
        expect = np.zeros(N)
        expect[0], expect[1] = 1 / a, -r / a
        np.testing.assert_allclose(inv[:, 0, 0], expect, rtol=0, atol=1e-14)


def _markov_mats(params):
    P, p = params["P"], params["p"]
    M = np.diag(1 - p) + np.diag(p) @ P
    return M, np.diag(p) @ P


def test_markov_closed_forms_all_outputs():
    """Geometric sojourns make the model a Markov chain with one-step matrix
    M = diag(1-p) + diag(p) P^emb, so psi(k) = M^{k-1} diag(p) P^emb (k >= 1),
    P(k) = M^k, g_D(k) = M_CC^{k-1} M_CD, S_D(k) = alpha_C M_CC^k 1,
    availability alpha M^k 1_U and renewal visits alpha sum_{l<=k} psi(l) I_B 1."""
    d, N = 5, 300
    q, params = synth.geometric_model(d, N, seed=11)
    M, J = _markov_mats(params)
    psi = oracle.inverse_left(synth.identity_minus(q))
    Pk = oracle.transition(psi, q)
    Mk = np.eye(d)
    psi_ref = [np.eye(d)]
    P_ref = [np.eye(d)]
    for k in range(1, N):
        psi_ref.append(Mk @ J)
        Mk = Mk @ M
        P_ref.append(Mk.copy())
    np.testing.assert_allclose(psi, np.array(psi_ref), atol=2e-14)
    np.testing.assert_allclose(Pk, np.array(P_ref), atol=2e-13)

    D = [3, 4]
    C = [0, 1, 2]
    alphaC = np.array([0.5, 0.3, 0.2])
    g, F, S = oracle.first_entrance(q, D, alphaC)
    Mcc, Mcd = M[np.ix_(C, C)], M[np.ix_(C, D)]
    Mp = np.eye(3)
    for k in range(N):
        if k == 0:
            np.testing.assert_allclose(g[0], 0.0, atol=0)
        else:
            np.testing.assert_allclose(g[k], Mp @ Mcd, atol=2e-14)
            Mp = Mp @ Mcc
        Sk = alphaC @ np.linalg.matrix_power(Mcc, k) @ np.ones(3)
        assert abs(S[k] - Sk) < 2e-13
        assert abs(F[k] + S[k] - 1.0) < 1e-15

    alpha = np.array([0.2, 0.2, 0.2, 0.2, 0.2])
    avail = oracle.occupation(Pk, alpha, C)
    for k in (0, 1, 7, 100, 299):
        ref = alpha @ np.linalg.matrix_power(M, k) @ np.isin(np.arange(d), C).astype(float)
        assert abs(avail[k] - ref) < 2e-13
    visits = oracle.renewal_visits(psi, alpha, [1, 4])
    IB1 = np.isin(np.arange(d), [1, 4]).astype(float)
    ref = np.cumsum([alpha @ psi_ref[k] @ IB1 for k in range(N)])
    np.testing.assert_allclose(visits, ref, atol=1e-12)


# ----------------------------------------------------------- algebra pins
def test_convolve_vs_numpy_polynomial_product():
    rng = np.random.default_rng(6)
    N = 37
    A = rng.standard_normal((N, 2, 3))
    B = rng.standard_normal((N, 3, 4))
    C = oracle.convolve(A, B)
    ref = np.zeros((N, 2, 4))
    for i in range(2):
        for j in range(4):
            for t in range(3):
                ref[:, i, j] += np.convolve(A[:, i, t], B[:, t, j])[:N]
    np.testing.assert_allclose(C, ref, rtol=1e-13, atol=1e-13)


def test_two_sided_inverse_and_residuals():
    q, _ = synth.weibull_model(6, 256, seed=7)
    A = synth.identity_minus(q)
    L = oracle.inverse_left(A)
    R = oracle.inverse_right(A)
    np.testing.assert_allclose(L, R, atol=1e-14)
    rl, rr = oracle.residuals(A, L)
    assert oracle.norm1_frob(rl) < 1e-13 and oracle.norm1_frob(rr) < 1e-12
    # sampled single-coefficient residual agrees with the full one
    for k in (0, 1, 100, 255):
        np.testing.assert_allclose(oracle.residual_left_at(A, L, k), rl[k], atol=1e-16)


def test_residual_entries_vs_numpy_polynomial_products():
    """rho_L(k)_ij = delta - sum_u (A_iu * psi_uj)(k) and rho_R(k)_ij =
    delta - sum_u (psi_iu * A_uj)(k), each 1-D convolution by np.convolve;
    integer entries make both sides exact.  A transposed operand or a
    dropped l = 0 term would fail here."""
    rng = np.random.default_rng(77)
    d, N = 3, 40
    A = rng.integers(-5, 6, size=(N, d, d)).astype(np.float64)
    P = rng.integers(-5, 6, size=(N, d, d)).astype(np.float64)
    for k in (0, 1, 17, N - 1):
        for i in range(d):
            for j in range(d):
                dl = 1.0 if (k == 0 and i == j) else 0.0
                wl = dl - sum(np.convolve(A[:, i, u], P[:, u, j])[k] for u in range(d))
                wr = dl - sum(np.convolve(P[:, i, u], A[:, u, j])[k] for u in range(d))
                assert oracle.residual_left_entry(A, P, k, i, j) == wl
                assert oracle.residual_right_entry(A, P, k, i, j) == wr


def test_norm1_frob_vs_numpy():
    """||X||_{1,N} with the Frobenius norm per coefficient: the sum over k of
    numpy's matrix Frobenius norm (a missing square root, or squares summed
    over k, would fail)."""
    rng = np.random.default_rng(78)
    X = rng.standard_normal((37, 4, 3))
    ref = sum(np.linalg.norm(X[k], "fro") for k in range(X.shape[0]))
    assert abs(oracle.norm1_frob(X) - ref) <= 1e-13 * ref
    Y = np.zeros((5, 2, 2))
    Y[2] = [[3.0, 0.0], [0.0, 4.0]]
    assert oracle.norm1_frob(Y) == 5.0


def test_prefix_exactness():
    """Proposition 2.3: the first N' coefficients depend only on A(0..N'-1)."""
    q, _ = synth.weibull_model(4, 200, seed=8)
    A = synth.identity_minus(q)
    full = oracle.inverse_left(A)
    pre = oracle.inverse_left(A[:50])
    assert np.array_equal(full[:50], pre)


def test_transition_rows_sum_to_one_and_equation_forms():
    """P = psi * Hbar satisfies P(k) 1 = 1 exactly (P 1 = s0 * psi * (e0 - q) 1) and
    the other form of Eq. (transition-discrete), P = Hbar + q * P."""
    q, _ = synth.weibull_model(5, 300, seed=9)
    psi = oracle.inverse_left(synth.identity_minus(q))
    P = oracle.transition(psi, q)
    np.testing.assert_allclose(P.sum(axis=2), 1.0, atol=2e-14)
    hb = oracle.hbar(q)
    rhs = oracle.convolve(q, P)
    rhs[:] += np.einsum("ki,ij->kij", hb, np.eye(5))
    np.testing.assert_allclose(P, rhs, atol=1e-14)
    assert np.all(np.diff(hb, axis=0) <= 1e-17) and np.all(hb[0] == 1.0)


def test_discrete_bounds():
    """q(0) = 0 allows at most one renewal per step: 0 <= psi_ij(k), sum_j psi_ij(k) <= 1
    for k >= 1; F_D is a nondecreasing probability."""
    q, _ = synth.weibull_model(6, 400, seed=10)
    psi = oracle.inverse_left(synth.identity_minus(q))
    assert psi[1:].min() > -1e-16
    assert psi[1:].sum(axis=2).max() < 1 + 1e-14
    g, F, S = oracle.first_entrance(q, [5], np.array([1, 0, 0, 0, 0.0]))
    assert np.all(np.diff(F) >= -1e-16) and F.min() >= 0 and F.max() <= 1 + 1e-14


def test_mean_value_rows_sum_to_one():
    """Mean-value solution K_h = (e0 - Qbar_h)^(-1) * [Hbar_h - 1/2 D+Q_h] (Eq. (mre-solution)
    with L = Hbar, L_h(0) = I) has unit row sums, since
    [Hbar_h(m) - 1/2 D+Q_h(m)] 1 = ((e0 - Qbar_h) * s0)(m) 1."""
    d, N, h = 4, 256, 0.05
    A, prm = synth.lognormal_model(d, N, seed=12, h=h)
    Qh = prm["Q"](h * np.arange(N + 1))
    Hbar = np.zeros((N, d, d))
    for m in range(N):
        Hbar[m] = np.diag(1.0 - Qh[m].sum(axis=1))
    dplus = Qh[1:N + 1] - Qh[0:N]
    rhs = Hbar - 0.5 * dplus
    K = oracle.convolve(oracle.inverse_left(A), rhs)
    np.testing.assert_allclose(K.sum(axis=2), 1.0, atol=1e-13)
    np.testing.assert_allclose(A[0], np.eye(d) - 0.5 * Qh[1], atol=0)


def test_perturbation_identity_and_bound():
    """Proposition 2.5 with q~ = fl32(q)."""
    q, _ = synth.weibull_model(3, 120, seed=13)
    qt = q.astype(np.float32).astype(np.float64)
    psi = oracle.inverse_left(synth.identity_minus(q))
    psit = oracle.inverse_left(synth.identity_minus(qt))
    lhs = psit - psi
    rhs = oracle.convolve(oracle.convolve(psit, qt - q), psi)
    np.testing.assert_allclose(lhs, rhs, atol=1e-15)
    bound = oracle.norm1_spec(psit) * oracle.norm1_spec(qt - q) * oracle.norm1_spec(psi)
    assert oracle.norm1_spec(lhs) <= bound


def test_residual_a_posteriori_bound():
    """Proposition 2.6 on a deliberately perturbed inverse, both sides."""
    rng = np.random.default_rng(14)
    q, _ = synth.weibull_model(3, 80, seed=14)
    A = synth.identity_minus(q)
    psi = oracle.inverse_left(A)
    pt = psi + 1e-5 * rng.standard_normal(psi.shape)
    rl, rr = oracle.residuals(A, pt)
    err = oracle.norm1_spec(psi - pt)
    for rho in (rl, rr):
        r = oracle.norm1_spec(rho)
        assert r < 1
        assert err <= r / (1 - r) * oracle.norm1_spec(pt) * (1 + 1e-9)


def test_spectral_norm_vs_numpy():
    rng = np.random.default_rng(15)
    assert abs(oracle.spectral_norm(np.diag([0.5, -3.0, 2.0])) - 3.0) < 1e-14
    u, v = rng.standard_normal(4), rng.standard_normal(3)
    assert abs(oracle.spectral_norm(np.outer(u, v)) - np.linalg.norm(u) * np.linalg.norm(v)) < 1e-12
    for _ in range(5):
        M = rng.standard_normal((6, 6))
        assert abs(oracle.spectral_norm(M) - np.linalg.norm(M, 2)) < 1e-9 * np.linalg.norm(M, 2)


# ---------------------------------------------------- the paper's examples
def test_paper_first_entrance_example():
    """Section 5.1 first-entrance example: direct-convolution discrepancy of the
    order of 1e-16 and cumulative probability 1 at the final time."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_first_entrance.json")))
    N = gold["N"]
    q = synth.poisson_paper_e4(N)
    D, C = [0], [1, 2]
    alphaC = np.array(gold["alpha_C"])
    g, F, S = oracle.first_entrance(q, D, alphaC)
    # renewal equation g = q_CD + q_CC * g solved forward (Section 4.1)
    qcc, qcd = q[:, C][:, :, C], q[:, C][:, :, D]
    gr = np.zeros((N, 2, 1))
    for k in range(N):
        gr[k] = qcd[k] + sum(qcc[l] @ gr[k - l] for l in range(1, k + 1))
    mass = np.einsum("c,kcd->k", alphaC, g)
    mass_r = np.einsum("c,kcd->k", alphaC, gr)
    assert np.max(np.abs(mass - mass_r)) <= 10 * gold["max_abs_discrepancy"]
    assert abs(F[-1] - 1.0) < 1e-6
    A_C = synth.identity_minus(qcc)
    rl, rr = oracle.residuals(A_C, oracle.inverse_left(A_C))
    assert oracle.norm1_spec(rl) <= 10 * gold["left_residual"]
    assert oracle.norm1_spec(rr) <= 10 * gold["right_residual"]


@pytest.mark.parametrize("N", [128, 512, 2048])
def test_paper_table4_residual_scale(N):
    """Table 4: residuals of an FP64 inverse of the horizon-scaling model are at
    rounding level and grow with N.  Each direct recursion satisfies its own
    defining equation coefficient by coefficient, so its own-side residual
    (left for the left recursion, right for Eq. (inverse-recursion)) must land
    on the scale of the FFT-Newton residuals the paper prints, within a factor
    4 (different summation orders), and the two recursions must agree to the
    paper's d_N scale."""
    gold = {int(r["N"]): r for r in json.load(open(os.path.join(GOLDEN, "paper_table4.json")))["rows"]}
    q = synth.gamma_paper_e1(N)
    A = synth.identity_minus(q)
    psi = oracle.inverse_left(A)
    psir = oracle.inverse_right(A)
    rl, _ = oracle.residuals(A, psi)
    _, rr = oracle.residuals(A, psir)
    assert oracle.norm1_spec(rl) <= 4 * gold[N]["newton_left_residual"]
    assert oracle.norm1_spec(rr) <= 4 * gold[N]["newton_right_residual"]
    fro = np.sqrt((psi ** 2).sum(axis=(1, 2)))
    dN = np.max(np.sqrt(((psir - psi) ** 2).sum(axis=(1, 2))) / np.maximum(fro, 2 ** -26.5))
    assert dN <= 4 * gold[N]["newton_dN"]


def _exponential_errors(h, T=40.0):
    """Max errors of the mean-value scheme against exp(G t) on [0, T] for the
    exponential benchmark: transition matrix (Frobenius), reliability and
    availability (Section 5, Table 5)."""
    import scipy.linalg as sl
    n = int(round(T / h)) + 1
    b = synth.exponential_benchmark(h, n)
    G, U, al = b["G"], b["U"], b["alpha"]
    K = oracle.mre_solve(b["Q"], b["Hbar"])
    KU = oracle.mre_solve(b["Q"][:, :3, :3], b["LU"])
    oneU = np.array([1.0, 1.0, 1.0, 0.0])
    EP = ER = EA = 0.0
    for m in range(n):
        Pex = sl.expm(G * m * h)  # the exact Markov solution (library matrix exponential)
        EP = max(EP, np.linalg.norm(Pex - K[m]))
        EA = max(EA, abs(al @ Pex @ oneU - al @ K[m] @ oneU))
        Rex = al[U] @ sl.expm(G[np.ix_(U, U)] * m * h) @ np.ones(3)
        ER = max(ER, abs(Rex - (al[U] @ KU[m])[0]))
    return EP, ER, EA


def test_paper_table5_mean_value_convergence():
    """Table 5: the mean-value discretisation Eq. (mre-discrete), solved as
    Eq. (mre-solution), of the exponential benchmark has the printed maximum
    errors on [0, 40] against exp(G t) for h = 0.4 .. 0.025 -- transition
    matrix, reliability (the up-state equation K_U = L_U + Q_UU * K_U with
    L_U = 1 - H_i) and availability -- and the printed observed orders."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_table5.json")))
    errs = [_exponential_errors(h) for h in gold["h"]]
    for (EP, ER, EA), gp, gr, ga in zip(errs, gold["E_P"], gold["E_R"], gold["E_A"]):
        assert abs(EP / gp - 1) < 1e-3 and abs(ER / gr - 1) < 1e-3 and abs(EA / ga - 1) < 1e-3
    for i in range(1, len(errs)):
        for j, key in enumerate(("order_P", "order_R", "order_A")):
            assert abs(np.log2(errs[i - 1][j] / errs[i][j]) - gold[key][i]) < 2e-3


def test_mean_value_terms_and_row_sums():
    """The mean-value terms of a linear kernel Q(t) = t C are Qbar_h(0) = hC/2,
    Qbar_h(m) = hC (m >= 1), Delta+ Q_h = hC; and the mean-value transition
    function K_h (L = Hbar_h) is stochastic: [Hbar_h - (1/2) Delta+ Q_h] 1 =
    ((e0 - Qbar_h) * s0) 1 with s0 the unit step, so K_h(k) 1 = 1 exactly."""
    h, n = 0.1, 7
    C = np.array([[0.0, 0.3], [0.2, 0.1]])
    Qs = h * np.arange(n + 1)[:, None, None] * C[None]
    _, dQp, Qbar = oracle.mean_value_terms(Qs)
    assert np.allclose(Qbar[0], h * C / 2) and np.allclose(Qbar[1:], h * C) and np.allclose(dQp, h * C)
    Qs, Hbar = synth.lognormal_samples(5, 400, seed=3, h=0.05)
    K = oracle.mre_solve(Qs, Hbar)
    assert np.abs(K.sum(axis=2) - 1.0).max() < 1e-12
    Pp = oracle.process_discretization(Qs, Hbar)
    assert np.abs(Pp.sum(axis=2) - 1.0).max() < 1e-12
