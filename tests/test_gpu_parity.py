"""GPU parity: libmrc (through the C ABI) against the FP64 oracle on the same
seeded inputs.

Tolerances:
* FP64 path: max_{k,i,j} |psi - psi_oracle| <= 1e-11 (absolute; every output
  is a probability or a bounded renewal density).
* mixed path: e_rel = sum_k ||psi(k) - psi_ref(k)||_F / sum_k ||psi_ref(k)||_F
  <= 1e-10 and max |rho_L| <= 1e-10.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_30379_gb300 import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-11
TOL_REL = 1e-10


@pytest.fixture(scope="module")
def mrc():
    from paper_2605_30379_gb300 import build
    build.build()
    from paper_2605_30379_gb300 import mrc as m
    m.load()
    return m


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def e_rel(got, ref):
    num = np.sqrt(((got - ref) ** 2).sum(axis=(1, 2))).sum()
    den = np.sqrt((ref ** 2).sum(axis=(1, 2))).sum()
    return num / den


# ------------------------------------------------------------- inverse FP64
@pytest.mark.parametrize("d,N,seed", [
    (4, 1024, 0),    # the small d=4 horizon-1024 Weibull workload
    (1, 1, 1), (1, 2, 1), (2, 3, 1), (3, 5, 2),   # degenerate / ragged horizons
    (3, 1000, 3), (5, 513, 4), (9, 300, 5),        # non power-of-two N, odd d
    (17, 700, 6), (40, 260, 7), (64, 130, 8),      # several product tiles, ragged
    (22, 600, 13), (24, 333, 14),                   # the 24 x 24 tile, full and ragged
    (16, 4096, 9),                                  # d=16 horizon-2^12 Weibull workload
])
def test_inverse_fp64_matches_oracle(mrc, d, N, seed):
    if d == 1:
        rng = np.random.default_rng(seed)
        q = np.zeros((N, 1, 1))
        q[1:, 0, 0] = rng.uniform(0, 1, N - 1) / max(1, N)
    else:
        q, _ = synth.weibull_model(d, N, seed=seed)
    A = synth.identity_minus(q)
    ref = oracle.inverse_left(A)
    psi = mrc.inverse(dev(A), prec="fp64").cpu().numpy()
    assert np.abs(psi - ref).max() <= TOL64


def test_inverse_fp64_general_A0_lognormal(mrc):
    """Mean-value reduction: A(0) = I - Q(h)/2 is not the identity."""
    A, _ = synth.lognormal_model(8, 1500, seed=10, h=0.05)
    ref = oracle.inverse_left(A)
    psi = mrc.inverse(dev(A), prec="fp64").cpu().numpy()
    assert np.abs(psi - ref).max() <= TOL64


def test_inverse_fp64_signed_dense(mrc):
    """A sequence with mixed signs and a dense non-identity A(0)."""
    rng = np.random.default_rng(11)
    d, N = 6, 777
    A = rng.standard_normal((N, d, d)) * (0.5 ** np.arange(N))[:, None, None] * 0.3
    A[0] += 2.0 * np.eye(d)
    ref = oracle.inverse_left(A)
    psi = mrc.inverse(dev(A), prec="fp64").cpu().numpy()
    assert np.abs(psi - ref).max() <= TOL64 * max(1.0, np.abs(ref).max())


def test_markov_closed_form_d16(mrc):
    """Geometric sojourns: psi(k) = M^{k-1} diag(p) P^emb."""
    d, N = 16, 4096
    q, prm = synth.geometric_model(d, N, seed=12)
    M = np.diag(1 - prm["p"]) + np.diag(prm["p"]) @ prm["P"]
    J = np.diag(prm["p"]) @ prm["P"]
    psi = mrc.inverse(dev(synth.identity_minus(q)), prec="fp64").cpu().numpy()
    Mk = np.eye(d)
    worst = 0.0
    for k in range(1, N):
        worst = max(worst, np.abs(psi[k] - Mk @ J).max())
        Mk = Mk @ M
    assert worst <= TOL64
    assert np.all(psi[0] == np.eye(d))


def test_singular_A0_reports_error(mrc):
    A = np.zeros((64, 3, 3))
    A[0] = [[1, 2, 3], [2, 4, 6], [0, 0, 1.0]]
    with pytest.raises(mrc.MrcError) as ei:
        mrc.inverse(dev(A), prec="fp64", report=True)
    assert ei.value.status == 2
    # the context stays usable after the error
    q, _ = synth.weibull_model(3, 64, seed=1)
    A2 = synth.identity_minus(q)
    psi = mrc.inverse(dev(A2), prec="fp64", report=True)[0].cpu().numpy()
    assert np.abs(psi - oracle.inverse_left(A2)).max() <= TOL64


# ------------------------------------------------- series Gauss-Jordan (App. D)
@pytest.mark.parametrize("d,N,seed", [
    (1, 1, 0), (1, 70, 1), (2, 1, 2), (2, 33, 3),   # degenerate and ragged horizons
    (3, 1000, 4), (4, 257, 5), (6, 2048, 6), (8, 513, 7), (13, 300, 8),
])
def test_inverse_gj_matches_oracle(mrc, d, N, seed):
    if d == 1:
        rng = np.random.default_rng(seed)
        q = np.zeros((N, 1, 1))
        q[1:, 0, 0] = rng.uniform(0, 1, N - 1) / max(1, N)
    else:
        q, _ = synth.weibull_model(d, N, seed=seed)
    A = synth.identity_minus(q)
    psi, rep = mrc.inverse_gj(dev(A), report=True)
    assert rep["levels"] == d
    assert np.abs(psi.cpu().numpy() - oracle.inverse_left(A)).max() <= TOL64


def test_inverse_gj_row_exchanges(mrc):
    """A(0) with a zero diagonal (a scaled permutation plus a small dense
    part): every column's pivot comes from another row, so the row exchanges
    of the augmented matrix are exercised; signed dense later coefficients."""
    rng = np.random.default_rng(21)
    d, N = 5, 600
    A = rng.standard_normal((N, d, d)) * (0.6 ** np.arange(N))[:, None, None] * 0.2
    perm = [2, 0, 4, 1, 3]
    A[0] = 0.05 * rng.standard_normal((d, d))
    np.fill_diagonal(A[0], 0.0)
    for i, j in enumerate(perm):
        A[0, i, j] = 2.0 + i
    ref = oracle.inverse_left(A)
    psi = mrc.inverse_gj(dev(A)).cpu().numpy()
    assert np.abs(psi - ref).max() <= TOL64 * max(1.0, np.abs(ref).max())


def test_inverse_gj_paper_scaling_kernels(mrc):
    """The kernels of the paper's scaling experiments (Section 5): s = 3 with
    shifted discrete Gamma sojourns at N = 2048, and the shifted Poisson
    state-dimension kernel at N = 256 for s = 2, 4, 6, 8; against the oracle,
    with left and right residuals in the range the paper reports for its
    accelerated inverses (Table 3: at most 5.2e-13)."""
    cases = [synth.gamma_paper_e1(2048)] + [synth.poisson_paper_e2(s, 256) for s in (2, 4, 6, 8)]
    for q in cases:
        A = synth.identity_minus(q)
        Ad = dev(A)
        psi = mrc.inverse_gj(Ad)
        assert np.abs(psi.cpu().numpy() - oracle.inverse_left(A)).max() <= TOL64
        _, _, r = mrc.residual(Ad, psi, sides=3, prec="fp64", want_rho=False)
        assert r["res_left_l1"] <= 1e-12 and r["res_right_l1"] <= 1e-12, r


def test_inverse_gj_singular_A0(mrc):
    A = np.zeros((64, 3, 3))
    A[0] = [[1, 2, 3], [2, 4, 6], [0, 0, 1.0]]
    with pytest.raises(mrc.MrcError) as ei:
        mrc.inverse_gj(dev(A), report=True)
    assert ei.value.status == 2
    psi = mrc.inverse_gj(dev(A))  # without a report: NaN output, status word read afterwards
    with pytest.raises(mrc.MrcError):
        mrc.sync_status()
    assert torch.isnan(psi).all()
    q, _ = synth.weibull_model(3, 64, seed=1)
    A2 = synth.identity_minus(q)
    psi2 = mrc.inverse_gj(dev(A2), report=True)[0].cpu().numpy()
    assert np.abs(psi2 - oracle.inverse_left(A2)).max() <= TOL64


def test_inverse_gj_long_horizon_matches_newton(mrc):
    """d = 4, N = 2^16 (two-pass transforms): Gauss-Jordan against FFT-Newton
    on the same input, the 4096-prefix against the oracle (Proposition 2.3),
    and sampled residual entries at k = N - 1 against the oracle's sums."""
    d, N = 4, 1 << 16
    q, _ = synth.weibull_model(d, N, seed=31)
    A = synth.identity_minus(q)
    Ad = dev(A)
    gj = mrc.inverse_gj(Ad)
    nw = mrc.inverse(Ad, prec="fp64")
    assert float((gj - nw).abs().max()) <= TOL64
    n = 4096
    assert np.abs(gj[:n].cpu().numpy() - oracle.inverse_left(A[:n])).max() <= TOL64
    g = gj.cpu().numpy()
    for i, j in ((0, 0), (3, 1), (2, 2)):
        assert abs(oracle.residual_left_entry(A, g, N - 1, i, j)) <= 1e-12


def test_bounded_wait_times_out_and_context_stays_usable(mrc):
    """Failure detection without a fault: the tensor-core kernels' bounded
    mbarrier wait, run on a barrier nothing arrives on, gives up after its
    spin limit and reports MRC_ERR_TIMEOUT through the status word; the status
    is cleared by the read and the context then still computes an inverse
    that matches the oracle."""
    import time
    t0 = time.perf_counter()
    mrc.selftest_timeout(spins=256)
    with pytest.raises(mrc.MrcError) as ei:
        mrc.sync_status()
    assert ei.value.status == 6
    assert time.perf_counter() - t0 < 30.0
    mrc.sync_status()  # cleared by the read
    q, _ = synth.weibull_model(5, 600, seed=24)
    A = synth.identity_minus(q)
    psi = mrc.inverse(dev(A), prec="fp64", report=True)[0].cpu().numpy()
    assert np.abs(psi - oracle.inverse_left(A)).max() <= TOL64


# ------------------------------------------------------------ inverse mixed
@pytest.mark.parametrize("d,N,seed", [(4, 1024, 0), (3, 777, 1), (16, 2048, 2), (33, 300, 3),
                                      (20, 1500, 4), (48, 2000, 5), (64, 1300, 6),
                                      (2, 1, 7), (40, 1, 8), (40, 2, 9), (5, 3, 10)])
def test_inverse_mixed_matches_oracle(mrc, d, N, seed):
    q, _ = synth.weibull_model(d, N, seed=seed)
    A = synth.identity_minus(q)
    ref = oracle.inverse_left(A)
    psi, rep = mrc.inverse(dev(A), prec="mixed", sweeps=1, target_residual=1e-10, report=True)
    psi = psi.cpu().numpy()
    assert e_rel(psi, ref) <= TOL_REL
    assert rep["res_max_abs"] <= TOL_REL


def test_inverse_mixed_lognormal_general_A0(mrc):
    A, _ = synth.lognormal_model(12, 1024, seed=4, h=0.05)
    ref = oracle.inverse_left(A)
    psi = mrc.inverse(dev(A), prec="mixed").cpu().numpy()
    assert e_rel(psi, ref) <= TOL_REL


# ------------------------------------------------------------------ residual
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_residual_matches_oracle(mrc, prec):
    rng = np.random.default_rng(20)
    q, _ = synth.weibull_model(5, 600, seed=20)
    A = synth.identity_minus(q)
    psi = oracle.inverse_left(A) + 1e-6 * rng.standard_normal(A.shape)
    rl_ref, rr_ref = oracle.residuals(A, psi)
    rl, rr, rep = mrc.residual(dev(A), dev(psi), sides=3, prec=prec)
    rl, rr = rl.cpu().numpy(), rr.cpu().numpy()
    assert np.abs(rl - rl_ref).max() <= 1e-12
    assert np.abs(rr - rr_ref).max() <= 1e-12
    assert abs(rep["res_left_l1"] - oracle.norm1_frob(rl_ref)) <= 1e-9 * oracle.norm1_frob(rl_ref)
    assert abs(rep["res_right_l1"] - oracle.norm1_frob(rr_ref)) <= 1e-9 * oracle.norm1_frob(rr_ref)
    assert abs(rep["res_max_abs"] - np.abs(rl_ref).max()) <= 1e-12


@pytest.mark.parametrize("prec,u", [("fp64", 2.0 ** -53), ("mixed", 2.0 ** -46)])
def test_fft_product_within_prop_2_1_bound(mrc, prec, u):
    """Prop 2.1 (Eq. (fft-forward-error)): a product C = A * B formed by
    zero-padded FFTs, per-frequency matrix products and an inverse FFT obeys
    ||C - C_fl||_{G,L} <= sqrt(L) ||A||_{G,L} ||B||_{G,L} delta_{L,s}.
    mrc_residual forms rho = e0 - A * B that way (L = 2 pow2ceil(N)), so
    rho's error bounds the product's on [0, N).  Small integer entries make
    the oracle's direct sum exact.  Readings of the model constants:
    sigma_L = 7 u log2 L (radix-2 FFT with accurately rounded twiddles),
    gamma_s = sqrt(2) (s + 2) u; u = 2^-53 for FP64 and 2^-46 for the
    double-float residual (a few 2^-48 roundings per operation).  The
    measured error must also stay far below the bound's order u sqrt(L)
    log2 L, so the check is not vacuous."""
    rng = np.random.default_rng(23)
    d, N = 7, 1000
    A = rng.integers(-8, 9, size=(N, d, d)).astype(np.float64)
    B = rng.integers(-8, 9, size=(N, d, d)).astype(np.float64)
    rl_ref, _ = oracle.residuals(A, B)  # exact: integers below 2^53
    rl, _, _ = mrc.residual(dev(A), dev(B), sides=1, prec=prec)
    err = np.sqrt(((rl.cpu().numpy() - rl_ref) ** 2).sum())
    L = 2 * (1 << (N - 1).bit_length())
    sig = 7 * u * np.log2(L)
    gam = np.sqrt(2.0) * (d + 2) * u
    beta = 2 * sig + sig ** 2 + gam * (1 + sig) ** 2
    delta = beta + sig * (1 + beta)
    norm_g = lambda X: np.sqrt((X ** 2).sum())
    bound = np.sqrt(L) * norm_g(A) * norm_g(B) * delta
    assert err <= bound, (err, bound)
    assert err <= 1e-2 * bound, (err, bound)


# ---------------------------------------------------------- derived outputs
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_transition_matches_oracle(mrc, prec):
    d, N = 6, 900
    q, _ = synth.weibull_model(d, N, seed=21)
    psi = oracle.inverse_left(synth.identity_minus(q))
    ref = oracle.transition(psi, q)
    P = mrc.transition(dev(psi), dev(q), prec=prec).cpu().numpy()
    assert np.abs(P - ref).max() <= TOL64
    assert np.abs(P.sum(axis=2) - 1.0).max() <= 1e-12


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("mixed", 1e-10)])
def test_first_entrance_matches_oracle(mrc, prec, tol):
    d, N = 7, 800
    q, _ = synth.weibull_model(d, N, seed=22)
    D = [2, 6]
    alphaC = np.array([0.1, 0.2, 0.3, 0.2, 0.2])
    g_ref, F_ref, S_ref = oracle.first_entrance(q, D, alphaC)
    g, F, S = mrc.first_entrance(dev(q), D, torch.tensor(alphaC), prec=prec)
    assert np.abs(g.cpu().numpy() - g_ref).max() <= tol
    assert np.abs(F.cpu().numpy() - F_ref).max() <= tol
    assert np.abs(S.cpu().numpy() - S_ref).max() <= tol


def test_paper_first_entrance_example(mrc):
    """Section 5.1 example: D = {1}, C = {2, 3}, alpha_C = (1, 0), N = 128."""
    q = synth.poisson_paper_e4(128)
    g_ref, F_ref, S_ref = oracle.first_entrance(q, [0], np.array([1.0, 0.0]))
    g, F, S = mrc.first_entrance(dev(q), [0], torch.tensor([1.0, 0.0]), prec="fp64")
    mass = g.cpu().numpy()[:, 0, 0]
    assert np.abs(mass - g_ref[:, 0, 0]).max() <= 1e-15
    assert abs(F.cpu().numpy()[-1] - 1.0) < 1e-6


def test_occupation_matches_oracle(mrc):
    d, N = 5, 400
    q, _ = synth.weibull_model(d, N, seed=23)
    psi = oracle.inverse_left(synth.identity_minus(q))
    P = oracle.transition(psi, q)
    alpha = np.array([0.3, 0.1, 0.2, 0.2, 0.2])
    ref = oracle.occupation(P, alpha, [0, 1, 3])
    got = mrc.occupation(dev(P), torch.tensor(alpha), [0, 1, 3]).cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-14


def test_batched_matches_single(mrc):
    models = synth.batch_models(n=6, seed=3, d_range=(3, 12), logN_range=(6.0, 9.0))
    As = [dev(m["A"]) for m in models]
    outs = mrc.inverse_batched(As, prec="fp64")
    for m, o in zip(models, outs):
        ref = oracle.inverse_left(m["A"])
        assert np.abs(o.cpu().numpy() - ref).max() <= TOL64


def test_batched_mixed_and_graph_replay(mrc):
    """Uneven d and non-power-of-two N in one captured batch; a second call
    with the same configuration replays the graph and must give the same bits."""
    models = synth.batch_models(n=10, seed=5, d_range=(3, 20), logN_range=(7.0, 10.5))
    As = [dev(m["A"]) for m in models]
    outs, reps = mrc.inverse_batched(As, prec="mixed", report=True)
    first = [o.clone() for o in outs]
    for m, o, r in zip(models, outs, reps):
        ref = oracle.inverse_left(m["A"])
        assert e_rel(o.cpu().numpy(), ref) <= TOL_REL
        assert r["sweeps"] == 1 and r["levels"] >= 1
    outs2 = mrc.inverse_batched(As, prec="mixed", outs=outs)
    torch.cuda.synchronize()
    for a, b in zip(first, outs2):
        assert torch.equal(a, b)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_waves_and_segment_groups(mrc, prec):
    """170 models (more than one segmented launch holds: 144) with d from 1 to
    40 and ragged N, on a context whose workspace cap splits them into several
    waves: every model against the oracle."""
    rng = np.random.default_rng(17)
    models = []
    for b in range(170):
        d = int(rng.integers(1, 41)) if b % 10 == 0 else int(rng.integers(1, 9))
        N = int(rng.integers(1, 300))
        q, _ = synth.weibull_model(d, N, seed=100 + b) if d > 1 else (None, None)
        if d == 1:
            q = np.zeros((N, 1, 1))
            q[1:, 0, 0] = rng.uniform(0, 1, N - 1) / max(1, N)
        models.append(synth.identity_minus(q))
    cap = 4 * max(mrc.workspace_bytes(a.shape[1], a.shape[0], prec) for a in models)
    ctx = mrc.create_context(max_workspace_bytes=cap + (1 << 20))
    try:
        As = [dev(a) for a in models]
        outs = mrc.inverse_batched(As, prec=prec, ctx=ctx)
        torch.cuda.synchronize()
        for a, o in zip(models, outs):
            ref = oracle.inverse_left(a)
            got = o.cpu().numpy()
            if prec == "fp64":
                assert np.abs(got - ref).max() <= TOL64
            else:
                assert e_rel(got, ref) <= TOL_REL
    finally:
        mrc.destroy_context(ctx)


def test_batched_reports_singular_model(mrc):
    q, _ = synth.weibull_model(3, 50, seed=1)
    good = synth.identity_minus(q)
    bad = np.zeros((40, 3, 3))
    bad[0] = [[1, 2, 3], [2, 4, 6], [0, 0, 1.0]]
    with pytest.raises(mrc.MrcError) as ei:
        mrc.inverse_batched([dev(good), dev(bad), dev(good)], prec="fp64", report=True)
    assert ei.value.status == 2
    outs = mrc.inverse_batched([dev(good), dev(good)], prec="fp64")
    for o in outs:
        assert np.abs(o.cpu().numpy() - oracle.inverse_left(good)).max() <= TOL64


@pytest.mark.parametrize("d,N", [(40, 300), (64, 200), (48, 513), (33, 129), (96, 100), (130, 33),
                                 (32, 300), (47, 200)])
def test_tensor_core_dd_residual_matches_oracle(mrc, d, N):
    """The double-float residual product for 32 <= d <= 512 runs as exact
    digit products on the tcgen05 tensor cores; both residuals must match
    the oracle's to 1e-12 (d = 33: padded tiles with a ragged edge; N = 129:
    a partial last pair range and the self-paired middle frequency; d = 96
    and 130: several 64 x 64 output tiles and K chunks, ragged; d = 32, 33,
    47, 48: two or three K chunks of 16 per frequency)."""
    rng = np.random.default_rng(d)
    q, _ = synth.weibull_model(d, N, seed=d)
    A = synth.identity_minus(q)
    psi = oracle.inverse_left(A) + 1e-6 * rng.standard_normal(A.shape)
    rl_ref, rr_ref = oracle.residuals(A, psi)
    rl, rr, _ = mrc.residual(dev(A), dev(psi), sides=3, prec="mixed")
    mrc.sync_status()
    assert np.abs(rl.cpu().numpy() - rl_ref).max() <= 1e-12
    assert np.abs(rr.cpu().numpy() - rr_ref).max() <= 1e-12


def test_mixed_inverse_d64_lognormal_prefix(mrc):
    """d = 64 mean-value Lognormal (the precision workload's shape) at a horizon
    the oracle finishes quickly: e_rel and the residual bound."""
    A, _ = synth.lognormal_model(64, 256, seed=0, h=0.05)
    ref = oracle.inverse_left(A)
    psi, rep = mrc.inverse(dev(A), prec="mixed", target_residual=1e-10, report=True)
    assert e_rel(psi.cpu().numpy(), ref) <= TOL_REL
    assert rep["res_max_abs"] <= TOL_REL


@pytest.mark.parametrize("d", [6, 12])
def test_two_pass_transforms_ragged_entries_match_oracle(mrc, d):
    """N = 5000: transforms of 2^12 and 2^13 points (two Stockham passes), a
    partial last Newton level and a ragged valid-row range; d = 6 leaves
    E = 36 entries (a partial chunk of 16), d = 12 E = 144 (9 chunks)."""
    q, _ = synth.weibull_model(d, 5000, seed=61 + d)
    A = synth.identity_minus(q)
    ref = oracle.inverse_left(A)
    p64 = mrc.inverse(dev(A), prec="fp64").cpu().numpy()
    pmx = mrc.inverse(dev(A), prec="mixed").cpu().numpy()
    mrc.sync_status()
    assert np.abs(p64 - ref).max() <= TOL64
    assert e_rel(pmx, ref) <= TOL_REL


@pytest.mark.parametrize("d,N", [(64, 700), (40, 1500), (70, 300)])
def test_mixed_inverse_product_tiles_match_oracle(mrc, d, N):
    """The FP32 product with 64 x 64 output tiles (the two frequencies of a
    pair on the two halves of the CTA) at several output tiles with ragged
    edges (d = 70) and one partial tile (d = 40)."""
    q, _ = synth.weibull_model(d, N, seed=70 + d)
    A = synth.identity_minus(q)
    ref = oracle.inverse_left(A)
    psi, rep = mrc.inverse(dev(A), prec="mixed", target_residual=1e-10, report=True)
    assert e_rel(psi.cpu().numpy(), ref) <= TOL_REL
    assert rep["res_max_abs"] <= TOL_REL


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("pinned", [True, False])
def test_inverse_from_host_buffers_matches_device_call(mrc, prec, pinned):
    """mrc_inverse_host uploads A in the row ranges the Newton levels read
    (overlapping the first levels) and copies psi back; it runs the same
    kernels as mrc_inverse, so the results agree, pinned or pageable, and
    match the oracle.  N = 3000 gives several upload ranges and a partial
    last one; two calls in a row reuse the context's copy stream."""
    q, _ = synth.weibull_model(12, 3000, seed=81)
    A = synth.identity_minus(q)
    ref = oracle.inverse_left(A)
    dev_psi = mrc.inverse(dev(A), prec=prec).cpu().numpy()
    A_host = torch.from_numpy(A)
    if pinned:
        A_host = A_host.pin_memory()
    for _ in range(2):
        out = torch.empty(A.shape, dtype=torch.float64)
        if pinned:
            out = out.pin_memory()
        got, rep = mrc.inverse_host(A_host, prec=prec, out=out, report=True)
        got = got.numpy()
        assert np.abs(got - dev_psi).max() <= 1e-13
        if prec == "fp64":
            assert np.abs(got - ref).max() <= TOL64
        else:
            assert e_rel(got, ref) <= TOL_REL


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("scheme", ["mean_value", "process"])
def test_mre_solve_matches_oracle(mrc, prec, scheme):
    """mrc_mre_solve (Section 4: Eq. (mre-solution) or Eq.
    (process-discretization)) against the oracle on Lognormal kernel samples:
    the transition function (L = Hbar, square) and a rectangular right-hand
    side, N = 700 (a partial last Newton level)."""
    Qs, Hbar = synth.lognormal_samples(6, 700, seed=91, h=0.05)
    rng = np.random.default_rng(92)
    Lr = rng.uniform(0, 1, (700, 6, 2))
    for L in (Hbar, Lr):
        ref = (oracle.mre_solve if scheme == "mean_value" else oracle.process_discretization)(Qs, L)
        got = mrc.mre_solve(dev(Qs), dev(L), scheme=scheme, prec=prec).cpu().numpy()
        mrc.sync_status()
        tol = 1e-11 if prec == "fp64" else 1e-10
        assert np.abs(got - ref).max() <= tol * max(1.0, np.abs(ref).max())


def test_mre_exponential_benchmark_n32768(mrc):
    """The exponential benchmark of Section 5 at N = 2^15, h = 0.005 on the
    GPU: maximum availability and reliability errors of the mean-value scheme
    against exp(G t) near the printed 2.53e-8 and 7.77e-8, of the process
    discretisation near 6.41e-5 and 1.86e-4 (tests/golden, three printed
    digits)."""
    n, h = 2 ** 15, 0.005
    b = synth.exponential_benchmark(h, n)
    G, U, al = b["G"], b["U"], b["alpha"]
    import scipy.linalg as sl
    # exact solution by repeated multiplication with exp(G h) (error ~ n u)
    step, stepU = sl.expm(G * h), sl.expm(G[np.ix_(U, U)] * h)
    Pex = np.empty((n, 4, 4)); Rex = np.empty(n)
    P, PU = np.eye(4), np.eye(3)
    for m in range(n):
        Pex[m] = P; Rex[m] = al[U] @ PU @ np.ones(3)
        P = P @ step; PU = PU @ stepU
    oneU = np.array([1.0, 1.0, 1.0, 0.0])
    Aex = np.einsum("i,mij,j->m", al, Pex, oneU)
    out = {}
    for scheme in ("mean_value", "process"):
        K = mrc.mre_solve(dev(b["Q"]), dev(b["Hbar"]), scheme=scheme, prec="fp64").cpu().numpy()
        KU = mrc.mre_solve(dev(b["Q"][:, :3, :3]), dev(b["LU"]), scheme=scheme, prec="fp64").cpu().numpy()
        out[scheme] = (np.abs(np.einsum("i,mij,j->m", al, K, oneU) - Aex).max(),
                       np.abs(np.einsum("i,mic->m", al[U], KU) - Rex).max())
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_exponential_benchmark.json")))
    for scheme in ("mean_value", "process"):
        ea, er = out[scheme]
        # three printed digits: within their rounding (0.5 %)
        assert abs(ea / gold[scheme]["availability"] - 1) < 5e-3, (scheme, ea)
        assert abs(er / gold[scheme]["reliability"] - 1) < 5e-3, (scheme, er)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_reward_matches_oracle(mrc, prec):
    """V = psi * r with a rectangular reward sequence (Eq. (reward)); the oracle
    side is its direct convolution, and V must solve V = r + q * V."""
    rng = np.random.default_rng(42)
    d, c, N = 6, 3, 700
    q, _ = synth.weibull_model(d, N, seed=42)
    psi = oracle.inverse_left(synth.identity_minus(q))
    r = rng.uniform(0, 1, (N, d, c))
    ref = oracle.convolve(psi, r)
    V = mrc.reward(dev(psi), dev(r), prec=prec).cpu().numpy()
    assert np.abs(V - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max())
    np.testing.assert_allclose(V, r + oracle.convolve(q, V), atol=1e-9)


def test_renewal_visits_matches_oracle(mrc):
    d, N = 5, 900
    q, _ = synth.weibull_model(d, N, seed=43)
    psi = oracle.inverse_left(synth.identity_minus(q))
    alpha = np.array([0.4, 0.1, 0.1, 0.2, 0.2])
    ref = oracle.renewal_visits(psi, alpha, [1, 3])
    got = mrc.renewal_visits(dev(psi), torch.tensor(alpha), [1, 3]).cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_autotuned_inverse_and_batch(mrc, tmp_path):
    """autotune=1 times the product-kernel candidates and the FFT plans (radix
    splits, entries per CTA) per shape on the call's stream; results stay
    within the parity gates and the choices are written to MRC_AUTOTUNE_CACHE
    when the context is destroyed (product choices 0..3, FFT plans below 512
    under keys with bit 62 set)."""
    import os
    cache = tmp_path / "tune.txt"
    os.environ["MRC_AUTOTUNE_CACHE"] = str(cache)
    try:
        q, _ = synth.weibull_model(40, 1500, seed=51)
        A = synth.identity_minus(q)
        ref = oracle.inverse_left(A)
        p64 = mrc.inverse(dev(A), prec="fp64", autotune=True).cpu().numpy()
        pmx = mrc.inverse(dev(A), prec="mixed", autotune=True).cpu().numpy()
        assert np.abs(p64 - ref).max() <= TOL64
        assert e_rel(pmx, ref) <= TOL_REL
        models = synth.batch_models(n=5, seed=52, d_range=(3, 40), logN_range=(7.0, 9.5))
        outs = mrc.inverse_batched([dev(m["A"]) for m in models], prec="mixed", autotune=True)
        for m, o in zip(models, outs):
            assert e_rel(o.cpu().numpy(), oracle.inverse_left(m["A"])) <= TOL_REL
        mrc.release()
        lines = cache.read_text().split()
        keys, picks = [int(k) for k in lines[0::2]], [int(c) for c in lines[1::2]]
        assert any(k >> 62 for k in keys) and any(not k >> 62 for k in keys)
        assert all(0 <= c <= (511 if k >> 62 else 4) for k, c in zip(keys, picks))
    finally:
        del os.environ["MRC_AUTOTUNE_CACHE"]
