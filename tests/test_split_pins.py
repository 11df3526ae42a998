"""Pins of the split-model oracle (Sec. 2.1.2, Fig. 3: a spatial and a colour
Normal-Wishart per component, one Dirichlet) against results other than
itself (CPU only).

The K = 1 fit converges in one iteration to the exact posterior of each
block, whose ELBO is then the exact log evidence of the two independent
blocks (closed form); log rho is the expectation of ln pi_k + ln N(s) +
ln N(c) under q, checked by Monte Carlo with scipy's Wishart, Gaussian and
Dirichlet samplers; the ELBO of a small mixture lies below its exact log
evidence by enumeration of every hard assignment.  A dropped block, a doubled
E[ln pi], the joint 6-D model in place of the split one, or a cross moment
leaking into a block fails one of them.
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy import stats
from scipy.special import logsumexp

from oracle import oracle as O
from oracle import split as SP
from tests import closed_forms as CF


def _prior(K, rng, nu0=7.5):
    A = rng.standard_normal((6, 6))
    W0 = A @ A.T / 6 + 0.5 * np.eye(6)
    return {"alpha0": 1.4, "beta0": 0.8, "nu0": nu0, "m0": rng.standard_normal((K, 6)), "W0": W0}


def _evidence_split(X, prior, k=0):
    m0, W0 = prior["m0"][k], prior["W0"]
    return (CF.nw_log_evidence(X[:, :3], m0[:3], prior["beta0"], W0[:3, :3], prior["nu0"])
            + CF.nw_log_evidence(X[:, 3:], m0[3:], prior["beta0"], W0[3:, 3:], prior["nu0"]))


def test_k1_converged_elbo_is_the_exact_evidence_of_both_blocks():
    rng = np.random.default_rng(21)
    prior = _prior(1, rng)
    X = rng.standard_normal((30, 6)) * 0.6 + 0.3
    elbo, S, _, _ = SP.cavi_frame(X, prior, np.zeros((1, 28)), 3)
    ev = _evidence_split(X, prior)
    assert abs(elbo[1] - ev) <= 1e-9 * abs(ev), (elbo, ev)
    assert abs(elbo[2] - ev) <= 1e-9 * abs(ev)
    q_s, q_c = SP.mstep(prior, S)
    for q, sl in ((q_s, slice(0, 3)), (q_c, slice(3, 6))):
        ref = CF.nw_posterior_centred(X[:, sl], prior["m0"][0, sl], prior["beta0"], prior["W0"][sl, sl],
                                      prior["nu0"])
        assert np.allclose(q["m"][0], ref["m"], rtol=1e-12, atol=1e-12)
        assert np.allclose(q["Winv"][0], ref["Winv"], rtol=1e-11, atol=1e-11)
        assert q["beta"][0] == ref["beta"] and q["nu"][0] == ref["nu"]
    # the joint 6-D model is a different model: its converged ELBO is not this evidence
    e_joint, _, _, _ = O.cavi_frame(X, prior, np.zeros((1, 28)), 2)
    assert abs(e_joint[1] - ev) > 1e-3 * abs(ev)


def test_k1_stream_carries_s_past_and_equals_the_batch_of_both_frames():
    """K = 1: every responsibility is 1, so a frame adds sum_n phi(x_n) (Eq. 3,
    phi = [1, x, upper(x x^T)] row-major) to S_past; two frames streamed
    through cavi_frame, the second from the first's S_past, give each block
    the conjugate posterior of both frames together (closed form)."""
    rng = np.random.default_rng(24)
    prior = _prior(1, rng)
    X1 = rng.standard_normal((20, 6)) * 0.5 + 0.2
    X2 = rng.standard_normal((25, 6)) * 0.7 - 0.1
    iu = np.triu_indices(6)

    def phi_sum(X):
        return np.concatenate([[X.shape[0]], X.sum(axis=0), (X.T @ X)[iu]])

    _, S1, _, _ = SP.cavi_frame(X1, prior, np.zeros((1, 28)), 2)
    _, S2, _, dS2 = SP.cavi_frame(X2, prior, S1, 2)
    assert np.allclose(dS2[0], phi_sum(X2), rtol=1e-12, atol=1e-9)
    assert np.allclose(S2[0], phi_sum(X1) + phi_sum(X2), rtol=1e-12, atol=1e-9)
    X = np.concatenate([X1, X2])
    q_s, q_c = SP.mstep(prior, S2)
    for q, sl in ((q_s, slice(0, 3)), (q_c, slice(3, 6))):
        ref = CF.nw_posterior_centred(X[:, sl], prior["m0"][0, sl], prior["beta0"], prior["W0"][sl, sl],
                                      prior["nu0"])
        assert np.allclose(q["m"][0], ref["m"], rtol=1e-12, atol=1e-12)
        assert np.allclose(q["Winv"][0], ref["Winv"], rtol=1e-10, atol=1e-10)


def _sample_nw(q, k, M, rng):
    """M draws of (mu, Lambda) from NW(m, beta, W, nu) of component k."""
    W = np.linalg.inv(q["Winv"][k])
    Lam = stats.wishart(df=q["nu"][k], scale=W).rvs(size=M, random_state=rng)
    C = np.linalg.cholesky(q["beta"][k] * Lam)              # beta Lambda = C C^T
    z = rng.standard_normal((M, 3, 1))
    mu = q["m"][k][None, :] + np.linalg.solve(np.transpose(C, (0, 2, 1)), z)[:, :, 0]
    return mu, Lam


def _log_normal(x, mu, Lam):
    d = x[None, :] - mu
    return 0.5 * np.linalg.slogdet(Lam)[1] - 1.5 * np.log(2 * np.pi) - 0.5 * np.einsum("mi,mij,mj->m", d, Lam, d)


def test_log_rho_is_the_expected_log_joint_by_monte_carlo():
    rng = np.random.default_rng(22)
    K = 3
    prior = _prior(K, rng)
    Xs = rng.standard_normal((40, 6)) * 0.8
    R = rng.dirichlet(np.ones(K), size=40)
    q_s, q_c = SP.mstep(prior, R.T @ SP.features(Xs))
    X = rng.standard_normal((3, 6)) * 0.7
    lr = SP.log_rho(X, q_s, q_c)
    M = 40000
    pis = rng.dirichlet(q_s["alpha"], size=M)
    for k in range(K):
        mu_s, L_s = _sample_nw(q_s, k, M, rng)
        mu_c, L_c = _sample_nw(q_c, k, M, rng)
        for n in range(X.shape[0]):
            v = np.log(pis[:, k]) + _log_normal(X[n, :3], mu_s, L_s) + _log_normal(X[n, 3:], mu_c, L_c)
            se = v.std() / np.sqrt(M)
            assert abs(v.mean() - lr[n, k]) < 5 * se, (k, n, v.mean(), lr[n, k], se)


def test_small_mixture_elbo_is_below_the_brute_force_evidence():
    rng = np.random.default_rng(23)
    K, N = 2, 6
    prior = _prior(K, rng)
    X = np.concatenate([rng.standard_normal((3, 6)) * 0.3 - 1.0, rng.standard_normal((3, 6)) * 0.3 + 1.0])
    terms = []
    for z in itertools.product(range(K), repeat=N):
        z = np.asarray(z)
        t = CF.dirichlet_multinomial_log(np.bincount(z, minlength=K), prior["alpha0"])
        for k in range(K):
            if np.any(z == k):
                t += _evidence_split(X[z == k], prior, k)
        terms.append(t)
    log_ev = float(logsumexp(terms))
    elbo, _, _, _ = SP.cavi_frame(X, prior, np.zeros((K, 28)), 40)
    assert np.all(elbo <= log_ev + 1e-9 * abs(log_ev)), (elbo.max(), log_ev)
    assert elbo[-1] > log_ev - 0.5 * abs(log_ev)


def test_cross_moments_do_not_enter_the_split_model():
    rng = np.random.default_rng(24)
    K = 5
    prior = _prior(K, rng)
    X = rng.standard_normal((60, 6))
    _, S, _, _ = SP.cavi_frame(X, prior, np.zeros((K, 28)), 2)
    S2 = S.copy()
    cross = [SP._upper_index(i, j, 6) for i in range(3) for j in range(3, 6)]
    assert len(cross) == 9
    S2[:, cross] += rng.standard_normal((K, 9)) * 5.0
    for a, b in zip(SP.mstep(prior, S), SP.mstep(prior, S2)):
        for key in a:
            assert np.array_equal(a[key], b[key])
    e1, _, _, _ = SP.cavi_frame(X[:20], prior, S, 2)
    e2, _, _, _ = SP.cavi_frame(X[:20], prior, S2, 2)
    assert np.array_equal(e1, e2)


def test_elbo_is_non_decreasing_and_counts_are_conserved():
    rng = np.random.default_rng(25)
    K, N = 4, 200
    prior = _prior(K, rng)
    X = rng.standard_normal((N, 6)) + np.repeat(rng.standard_normal((4, 6)) * 2, N // 4, axis=0)
    elbo, S, lse, dS = SP.cavi_frame(X, prior, np.zeros((K, 28)), 8)
    assert np.all(np.diff(elbo) >= -1e-9 * abs(elbo[-1])), elbo
    assert abs(dS[:, 0].sum() - N) <= 1e-9 * N
    assert np.allclose(S, dS)
    _, _, R = SP.estep_stats(X, *SP.mstep(prior, np.zeros((K, 28))))
    assert np.allclose(R.sum(axis=1), 1.0, atol=1e-12)
