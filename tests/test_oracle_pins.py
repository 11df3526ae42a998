"""Pins of the FP64 oracle against results other than itself (CPU only).

Each test fixes one part of the oracle to something the mathematics
determines independently of its code: closed forms of the conjugate
Normal-Wishart model, brute-force enumeration, Monte Carlo expectations
drawn by library samplers, special-function tables and invariants.  A
plausible mistake anywhere in the oracle (a dropped term of log rho, a wrong
sign in a KL, a transposed statistic, a wrong effective prior in the stream)
fails at least one of them.
"""
from __future__ import annotations

import math
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest
from scipy import stats
from scipy.special import digamma as sp_digamma, logsumexp, multigammaln, softmax

from oracle import oracle as O
from paper_2603_08499_gb300 import synth
from tests import closed_forms as CF

GOLDEN = Path(__file__).resolve().parent / "golden"
D = 6


def _random_prior(K, rng, D=6, nu0=None):
    A = rng.standard_normal((D, D))
    W0 = A @ A.T / D + 0.5 * np.eye(D)
    return {"alpha0": 1.3, "beta0": 0.7, "nu0": float(nu0 if nu0 else D + 2.5),
            "m0": rng.standard_normal((K, D)), "W0": W0}


def _random_post(K, rng, prior, N=30):
    """A posterior with distinct parameters per component: prior (+) random soft stats."""
    X = rng.standard_normal((N, prior["m0"].shape[1])) * 0.7
    R = rng.dirichlet(np.ones(K), size=N)
    S = R.T @ CF.features(X)
    return O.mstep(prior, S)


# ---- special functions -------------------------------------------------------

def test_digamma_golden_values():
    gamma = 0.57721566490153286060651209008240243
    ln2 = math.log(2.0)
    rows = [l.split(None, 1) for l in (GOLDEN / "digamma_special_values.txt").read_text().splitlines()
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 8
    for x, expr in rows:
        terms = expr.replace(" ", "").replace("-gamma", "").replace("-2*ln2", "")
        rational = sum((Fraction(t) for t in terms.split("+") if t), Fraction(0))
        want = -gamma - (2 * ln2 if "ln2" in expr else 0.0) + float(rational)
        assert abs(O.digamma(float(x)) - want) <= 2e-15 * max(1.0, abs(want)), (x, expr)


def test_digamma_and_mvgamma_vs_scipy():
    xs = np.concatenate([np.linspace(0.05, 30, 300), np.geomspace(30, 1e7, 50)])
    for x in xs:
        assert abs(O.digamma(x) - sp_digamma(x)) <= 4e-15 * max(1.0, abs(sp_digamma(x)))
    for a in [2.6, 3.0, 4.5, 10.25, 1e3, 5e5]:
        assert abs(O.lmvgamma(6, a) - multigammaln(a, 6)) <= 1e-13 * max(1.0, abs(multigammaln(a, 6)))


# ---- K = 1: the update is exact conjugate inference ---------------------------

def test_closed_form_helpers_agree():
    """The evidence closed form used below equals the chain rule of Student-t
    posterior predictives (scipy), so it is itself pinned."""
    rng = np.random.default_rng(3)
    pr = _random_prior(1, rng)
    X = rng.standard_normal((12, D))
    a = CF.nw_log_evidence(X, pr["m0"][0], pr["beta0"], pr["W0"], pr["nu0"])
    b = CF.nw_log_evidence_sequential(X, pr["m0"][0], pr["beta0"], pr["W0"], pr["nu0"])
    assert abs(a - b) <= 1e-10 * abs(a)


@pytest.mark.parametrize("N", [1, 7, 60])
def test_k1_posterior_and_elbo_equal_exact_evidence(N):
    rng = np.random.default_rng(10 + N)
    pr = _random_prior(1, rng)
    X = rng.standard_normal((N, D)) * 0.5 + 0.3
    elbo, S, lse, dS = O.cavi_frame(X, pr, np.zeros((1, 28)), 3)
    post = O.mstep(pr, S)
    ref = CF.nw_posterior_centred(X, pr["m0"][0], pr["beta0"], pr["W0"], pr["nu0"])
    assert np.allclose(post["m"][0], ref["m"], rtol=1e-12, atol=1e-13)
    assert np.allclose(post["Winv"][0], ref["Winv"], rtol=1e-11, atol=1e-12)
    assert post["beta"][0] == pytest.approx(ref["beta"], rel=1e-15)
    assert post["nu"][0] == pytest.approx(ref["nu"], rel=1e-15)
    assert post["alpha"][0] == pytest.approx(pr["alpha0"] + N, rel=1e-15)
    ev = CF.nw_log_evidence(X, pr["m0"][0], pr["beta0"], pr["W0"], pr["nu0"])
    # the bound is tight at the exact posterior: iterations 1 and 2
    assert abs(elbo[1] - ev) <= 1e-11 * abs(ev)
    assert abs(elbo[2] - ev) <= 1e-11 * abs(ev)
    assert elbo[0] <= ev + 1e-9 * abs(ev)
    assert np.allclose(dS[0, 0], N) and np.allclose(S, dS)


def test_streaming_k1_equals_batch_posterior():
    """Replay-free accumulation (Alg. 1): two frames in sequence give the batch
    posterior, and frame 2's bound equals ln p(X2 | X1)."""
    rng = np.random.default_rng(5)
    pr = _random_prior(1, rng)
    X1 = rng.standard_normal((25, D))
    X2 = rng.standard_normal((18, D)) + 0.4
    _, S1, _, _ = O.cavi_frame(X1, pr, np.zeros((1, 28)), 2)
    e2, S2, _, _ = O.cavi_frame(X2, pr, S1, 2)
    post = O.mstep(pr, S2)
    ref = CF.nw_posterior_centred(np.vstack([X1, X2]), pr["m0"][0], pr["beta0"], pr["W0"], pr["nu0"])
    assert np.allclose(post["Winv"][0], ref["Winv"], rtol=1e-11)
    assert np.allclose(post["m"][0], ref["m"], rtol=1e-12)
    ev12 = CF.nw_log_evidence(np.vstack([X1, X2]), pr["m0"][0], pr["beta0"], pr["W0"], pr["nu0"])
    ev1 = CF.nw_log_evidence(X1, pr["m0"][0], pr["beta0"], pr["W0"], pr["nu0"])
    assert abs(e2[1] - (ev12 - ev1)) <= 1e-10 * abs(ev12)


def test_hard_assignment_mstep_is_per_cluster_conjugate_update():
    rng = np.random.default_rng(6)
    K = 4
    pr = _random_prior(K, rng)
    X = rng.standard_normal((40, D))
    z = rng.integers(0, K, 40)
    R = np.eye(K)[z]
    post = O.mstep(pr, R.T @ CF.features(X))
    for k in range(K):
        ref = CF.nw_posterior_centred(X[z == k], pr["m0"][k], pr["beta0"], pr["W0"], pr["nu0"])
        assert np.allclose(post["Winv"][k], ref["Winv"], rtol=1e-11, atol=1e-12)
        assert np.allclose(post["m"][k], ref["m"], rtol=1e-12, atol=1e-13)


# ---- expectations of compute_elbo_delta and the KL terms (Monte Carlo) --------

def _sample_nw(post, k, n, rng):
    Lam = stats.wishart(df=post["nu"][k], scale=np.linalg.inv(post["Winv"][k])).rvs(size=n, random_state=rng)
    mus = np.empty((n, D))
    for i in range(n):
        mus[i] = rng.multivariate_normal(post["m"][k], np.linalg.inv(post["beta"][k] * Lam[i]))
    return mus, Lam


def test_log_rho_matches_monte_carlo_expectation():
    """log rho_nk = E_q[ln pi_k + ln N(x_n | mu_k, Lambda_k^-1)] (Alg. 1 compute_elbo_delta)."""
    rng = np.random.default_rng(7)
    K = 3
    pr = _random_prior(K, rng)
    post = _random_post(K, rng, pr, N=12)
    X = rng.standard_normal((4, D)) * 0.6
    lr = O.log_rho(X, post)
    n_mc = 4000
    pis = rng.dirichlet(post["alpha"], size=n_mc)
    for k in range(K):
        mus, Lam = _sample_nw(post, k, n_mc, rng)
        for n in range(X.shape[0]):
            d = X[n] - mus
            quad = np.einsum("si,sij,sj->s", d, Lam, d)
            ld = np.linalg.slogdet(Lam)[1]
            v = np.log(pis[:, k]) + 0.5 * ld - 0.5 * D * np.log(2 * np.pi) - 0.5 * quad
            se = v.std() / math.sqrt(n_mc)
            assert abs(lr[n, k] - v.mean()) < 5 * se + 1e-3, (n, k, lr[n, k], v.mean(), se)


def test_kl_nw_matches_monte_carlo_and_vanishes_at_equality():
    rng = np.random.default_rng(8)
    K = 2
    pr = _random_prior(K, rng)
    q = _random_post(K, rng, pr, N=20)
    p = O.mstep(pr, np.zeros((K, 28)))
    for k in range(K):
        assert abs(O.kl_nw(p, p, k)) < 1e-10
        n_mc = 3000
        mus, Lam = _sample_nw(q, k, n_mc, rng)

        def logpdf(par, mu, L):
            lw = stats.wishart(df=par["nu"][k], scale=np.linalg.inv(par["Winv"][k])).logpdf(L)
            ln = stats.multivariate_normal(par["m"][k], np.linalg.inv(par["beta"][k] * L)).logpdf(mu)
            return lw + ln

        v = np.array([logpdf(q, mus[i], Lam[i]) - logpdf(p, mus[i], Lam[i]) for i in range(n_mc)])
        se = v.std() / math.sqrt(n_mc)
        assert abs(O.kl_nw(q, p, k) - v.mean()) < 5 * se + 1e-3


def test_kl_dirichlet_matches_monte_carlo():
    rng = np.random.default_rng(9)
    a = np.array([1.5, 7.0, 3.2, 0.9])
    a0 = np.array([1.0, 1.0, 2.0, 0.5])
    assert abs(O.kl_dir(a, a)) < 1e-12
    s = rng.dirichlet(a, size=200000)
    v = stats.dirichlet(a).logpdf(s.T) - stats.dirichlet(a0).logpdf(s.T)
    assert abs(O.kl_dir(a, a0) - v.mean()) < 5 * v.std() / math.sqrt(s.shape[0])


# ---- responsibilities and statistics ------------------------------------------

def test_responsibilities_are_softmax_of_log_rho_and_stats_are_eq3():
    """R = softmax_k log rho (library), Delta S = R^T S_u (Eq. 3) equals the
    materialise-then-reduce form of Eqs. 1-2 over batches of B points."""
    rng = np.random.default_rng(11)
    K = 5
    pr = _random_prior(K, rng)
    post = _random_post(K, rng, pr)
    X = rng.standard_normal((1200, D)) * 0.8
    lse, dS, R = O.estep_stats(X, post, want_R=True)
    lr = O.log_rho(X, post)
    assert np.allclose(R, softmax(lr, axis=1), rtol=1e-12, atol=1e-300)
    assert np.allclose(lse, logsumexp(lr, axis=1), rtol=1e-13)
    Su = CF.features(X)
    B = 500
    acc = np.zeros_like(dS)
    for b0 in range(0, X.shape[0], B):       # Eq. 1 then Eq. 2 per batch
        dstar = R[b0:b0 + B, :, None] * Su[b0:b0 + B, None, :]
        acc += dstar.sum(axis=0)
    assert np.allclose(dS, acc, rtol=1e-12, atol=1e-10)
    # invariants of any responsibilities
    assert np.allclose(R.sum(axis=1), 1.0, rtol=0, atol=1e-13)
    assert dS[:, 0].sum() == pytest.approx(X.shape[0], rel=1e-13)
    assert np.allclose(dS[:, 1:7].sum(axis=0), X.sum(axis=0), rtol=1e-12, atol=1e-9)
    iu = np.triu_indices(D)
    assert np.allclose(dS[:, 7:].sum(axis=0), (X.T @ X)[iu], rtol=1e-12)


def test_bruteforce_evidence_bounds_every_elbo():
    """ELBO_t <= ln p(X), the exact evidence by enumerating all K^N assignments."""
    rng = np.random.default_rng(12)
    for K, N in [(2, 7), (3, 5)]:
        pr = {"alpha0": 1.0, "beta0": 1.0, "nu0": 8.0, "m0": rng.uniform(-1, 1, (K, D)), "W0": 4.0 * np.eye(D)}
        X = rng.uniform(-1, 1, (N, D))
        ev = CF.mixture_log_evidence_bruteforce(X, pr)
        elbo, _, _, _ = O.cavi_frame(X, pr, np.zeros((K, 28)), 12)
        assert np.all(elbo <= ev + 1e-9 * abs(ev)), (elbo, ev)
        assert np.all(np.diff(elbo) >= -1e-9 * abs(elbo[-1]))
        # the converged bound is close to (within a few nats of) the evidence
        assert ev - elbo[-1] < 5.0


def test_bruteforce_evidence_k1_equality():
    rng = np.random.default_rng(13)
    pr = {"alpha0": 1.0, "beta0": 1.0, "nu0": 8.0, "m0": rng.uniform(-1, 1, (1, D)), "W0": 4.0 * np.eye(D)}
    X = rng.uniform(-1, 1, (6, D))
    ev = CF.mixture_log_evidence_bruteforce(X, pr)
    elbo, _, _, _ = O.cavi_frame(X, pr, np.zeros((1, 28)), 2)
    assert abs(elbo[1] - ev) < 1e-11 * abs(ev)


# ---- whole-iteration properties ------------------------------------------------

def test_elbo_non_decreasing_on_mixture_workload():
    X, pr = synth.c1_workload(N=3000, K=120)
    elbo, S, _, _ = O.cavi_frame(X, pr, np.zeros((120, 28)), 15)
    assert np.all(np.diff(elbo) >= -1e-10 * abs(elbo[-1]))
    assert S[:, 0].sum() == pytest.approx(3000, rel=1e-12)


def test_empty_frame_keeps_prior_and_zero_elbo():
    rng = np.random.default_rng(14)
    pr = _random_prior(3, rng)
    S0 = np.abs(rng.standard_normal((3, 28))) * 0   # empty history
    elbo, S, lse, dS = O.cavi_frame(np.zeros((0, D)), pr, S0, 2)
    assert np.all(np.abs(elbo) < 1e-12) and np.all(S == 0.0) and np.all(dS == 0.0)


def test_affine_equivariance():
    """x -> s x + o with m0 -> s m0 + o, W0 -> W0 / s^2 leaves R unchanged and
    shifts the ELBO by -N D ln s (pins the frame independence of every term)."""
    rng = np.random.default_rng(15)
    K, N = 6, 300
    X, pr = synth.c1_workload(seed=3, N=N, K=K)
    s, o = 2.5, rng.standard_normal(D)
    pr2 = dict(pr, m0=pr["m0"] * s + o, W0=pr["W0"] / s**2)
    e1, S1, l1, _ = O.cavi_frame(X, pr, np.zeros((K, 28)), 4)
    e2, S2, l2, _ = O.cavi_frame(X * s + o, pr2, np.zeros((K, 28)), 4)
    assert np.allclose(S1[:, 0], S2[:, 0], rtol=1e-9, atol=1e-9)
    assert np.allclose(e2, e1 - N * D * math.log(s), rtol=1e-10)
    assert np.allclose(l2, l1 - D * math.log(s), rtol=1e-9, atol=1e-9)


def test_point_permutation_invariance():
    X, pr = synth.c1_workload(seed=5, N=800, K=30)
    perm = np.random.default_rng(0).permutation(800)
    e1, S1, _, _ = O.cavi_frame(X, pr, np.zeros((30, 28)), 3)
    e2, S2, _, _ = O.cavi_frame(X[perm], pr, np.zeros((30, 28)), 3)
    assert np.allclose(e1, e2, rtol=1e-12)
    assert np.allclose(S1, S2, rtol=1e-9, atol=1e-9)


def test_component_permutation_invariance():
    X, pr = synth.c1_workload(seed=6, N=600, K=25)
    perm = np.random.default_rng(1).permutation(25)
    e1, S1, _, _ = O.cavi_frame(X, pr, np.zeros((25, 28)), 3)
    e2, S2, _, _ = O.cavi_frame(X, dict(pr, m0=pr["m0"][perm]), np.zeros((25, 28)), 3)
    assert np.allclose(e1, e2, rtol=1e-12)
    assert np.allclose(S1[perm], S2, rtol=1e-9, atol=1e-9)


def test_elbo_entry_matches_update_trace():
    """or_elbo on the effective prior equals the first entry of the trace."""
    X, pr = synth.c1_workload(seed=7, N=500, K=20)
    _, S1, _, _ = O.cavi_frame(X[:250], pr, np.zeros((20, 28)), 3)
    e, _, _, _ = O.cavi_frame(X[250:], pr, S1, 2)
    assert O.elbo(X[250:], pr, S1) == pytest.approx(e[0], rel=1e-13)


# ---------------------------------------------------------------------------
# proposal network oracle (FP64): the backward pass against central finite
# differences of the forward pass, and closed forms of the loss


def _mlp_case(seed=0, B=6):
    from oracle import mlp as M
    rng = np.random.default_rng(seed)
    theta = np.concatenate([rng.normal(0, 1 / np.sqrt(s[-1]) if len(s) == 2 else 0.1, int(np.prod(s))).ravel()
                            for s in M.SHAPES])
    x = rng.uniform(-1, 1, (B, 6))
    q = rng.dirichlet(np.full(1024, 0.05), size=B)
    return M, theta, x, q


def test_mlp_gradient_matches_central_differences():
    M, theta, x, q = _mlp_case()
    g = M.grad(theta, x, q)
    rng = np.random.default_rng(1)
    # a coordinate sample from every parameter block plus one random direction
    sizes = [int(np.prod(s)) for s in M.SHAPES]
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    coords = np.concatenate([s + rng.choice(n, min(n, 40), replace=False) for s, n in zip(starts, sizes)])
    eps = 1e-6
    h1, h2, _ = M.forward(theta, x)
    # keep the sample away from ReLU kinks: no pre-activation within the step
    assert np.min(np.abs(h1[h1 > 0])) > 1e-4 and np.min(np.abs(h2[h2 > 0])) > 1e-4
    for i in coords:
        e = np.zeros_like(theta)
        e[i] = eps
        fd = (M.loss(theta + e, x, q) - M.loss(theta - e, x, q)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-9, (i, fd, g[i])
    v = rng.normal(size=theta.shape)
    v /= np.linalg.norm(v)
    fd = (M.loss(theta + eps * v, x, q) - M.loss(theta - eps * v, x, q)) / (2 * eps)
    assert abs(fd - g @ v) <= 1e-6 * abs(g @ v)


def test_mlp_loss_closed_forms():
    M, theta, x, q = _mlp_case(seed=2)
    # zero output layer: uniform softmax, loss = ln 1024 for any normalised q
    z0 = theta.copy()
    off = sum(int(np.prod(s)) for s in M.SHAPES[:4])
    z0[off:] = 0.0
    assert abs(M.loss(z0, x, q) - np.log(1024.0)) <= 1e-12
    # the output-bias gradient is the mean of softmax - q, which sums to 0
    g = M.grad(theta, x, q)
    assert abs(g[-1024:].sum()) <= 1e-12
    # loss >= entropy of q (Gibbs), equality only at softmax = q
    ent = -(q * np.log(np.where(q > 0, q, 1.0))).sum() / x.shape[0]
    assert M.loss(theta, x, q) >= ent


def test_top4_and_nearest_centroid_tie_rules():
    from oracle import mlp as M
    z = np.array([[1.0, 3.0, 3.0, 0.0, 3.0, 2.0, 3.0]])
    assert list(M.top4(z)[0]) == [1, 2, 4, 6]
    rng = np.random.default_rng(3)
    z = rng.integers(0, 5, (50, 40)).astype(float)
    t = M.top4(z)
    for row, sel in zip(z, t):
        # brute force: the 4 smallest (-value, index) pairs
        ref = sorted(range(len(row)), key=lambda j: (-row[j], j))[:4]
        assert list(sel) == ref
    c = np.array([[0.0, 0, 0, 0, 0, 0], [2.0, 0, 0, 0, 0, 0], [1.0, 0, 0, 0, 0, 0]])
    p = np.array([[0.5, 0, 0, 0, 0, 0], [1.5, 0, 0, 0, 0, 0], [3.0, 0, 0, 0, 0, 0]])
    a, _ = M.nearest_centroid(p, c)
    assert list(a) == [0, 1, 1]
