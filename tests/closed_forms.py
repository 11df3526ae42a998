"""Closed forms and brute-force references used to pin the oracle.

These are textbook results about the conjugate Normal-Wishart model that do
not go through the oracle's code: the exact posterior in centred (scatter
matrix) form, the exact log marginal likelihood, and the exact log evidence
of a small mixture by enumerating every hard assignment.
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy.special import gammaln, logsumexp, multigammaln


def nw_posterior_centred(X: np.ndarray, m0, beta0, W0, nu0):
    """Exact NW posterior after observing X (n x D), centred form:
    x_bar, scatter C = sum (x - x_bar)(x - x_bar)^T,
    W_n^-1 = W0^-1 + C + beta0 n / (beta0 + n) (x_bar - m0)(x_bar - m0)^T."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, len(m0))
    n = X.shape[0]
    W0inv = np.linalg.inv(W0)
    if n == 0:
        return {"beta": beta0, "nu": nu0, "m": np.array(m0, dtype=float), "Winv": W0inv}
    xb = X.mean(axis=0)
    C = (X - xb).T @ (X - xb)
    d = (xb - m0)[:, None]
    return {"beta": beta0 + n, "nu": nu0 + n, "m": (beta0 * np.asarray(m0) + n * xb) / (beta0 + n),
            "Winv": W0inv + C + beta0 * n / (beta0 + n) * (d @ d.T)}


def nw_log_evidence(X: np.ndarray, m0, beta0, W0, nu0) -> float:
    """ln p(X) under x ~ N(mu, Lambda^-1), (mu, Lambda) ~ NW(m0, beta0, W0, nu0):
    -(nD/2) ln pi + ln Gamma_D(nu_n/2) - ln Gamma_D(nu0/2)
    + (nu0/2) ln|W0^-1| - (nu_n/2) ln|W_n^-1| + (D/2) ln(beta0/beta_n)."""
    D = len(m0)
    X = np.asarray(X, dtype=np.float64).reshape(-1, D)
    n = X.shape[0]
    if n == 0:
        return 0.0
    post = nw_posterior_centred(X, m0, beta0, W0, nu0)
    ld0 = np.linalg.slogdet(np.linalg.inv(W0))[1]
    ldn = np.linalg.slogdet(post["Winv"])[1]
    return float(-0.5 * n * D * np.log(np.pi) + multigammaln(0.5 * post["nu"], D) - multigammaln(0.5 * nu0, D)
                 + 0.5 * nu0 * ld0 - 0.5 * post["nu"] * ldn + 0.5 * D * np.log(beta0 / post["beta"]))


def nw_log_evidence_sequential(X: np.ndarray, m0, beta0, W0, nu0) -> float:
    """The same evidence by the chain rule: sum_i ln p(x_i | x_<i) with the
    multivariate Student-t posterior predictive (scipy.stats.multivariate_t)."""
    from scipy.stats import multivariate_t
    D = len(m0)
    X = np.asarray(X, dtype=np.float64).reshape(-1, D)
    tot = 0.0
    for i in range(X.shape[0]):
        p = nw_posterior_centred(X[:i], m0, beta0, W0, nu0)
        dof = p["nu"] - D + 1
        shape = p["Winv"] * (p["beta"] + 1) / (p["beta"] * dof)
        tot += multivariate_t(loc=p["m"], shape=shape, df=dof).logpdf(X[i])
    return float(tot)


def dirichlet_multinomial_log(counts, alpha0: float) -> float:
    """ln p(z) of one ordered assignment with cluster counts under Dir(alpha0 1_K)."""
    counts = np.asarray(counts, dtype=np.float64)
    K = counts.size
    n = counts.sum()
    return float(gammaln(K * alpha0) - gammaln(n + K * alpha0) + np.sum(gammaln(counts + alpha0) - gammaln(alpha0)))


def mixture_log_evidence_bruteforce(X: np.ndarray, prior: dict) -> float:
    """Exact ln p(X) of the Bayesian mixture by summing over all K^N hard
    assignments z: ln sum_z p(z) prod_k p(X_{z=k})."""
    X = np.asarray(X, dtype=np.float64)
    N = X.shape[0]
    m0 = np.asarray(prior["m0"])
    K = m0.shape[0]
    terms = []
    for z in itertools.product(range(K), repeat=N):
        z = np.asarray(z)
        counts = np.bincount(z, minlength=K)
        t = dirichlet_multinomial_log(counts, prior["alpha0"])
        for k in range(K):
            t += nw_log_evidence(X[z == k], m0[k], prior["beta0"], prior["W0"], prior["nu0"])
        terms.append(t)
    return float(logsumexp(terms))


def features(X: np.ndarray) -> np.ndarray:
    """Unsummed statistics S_u = [1, x, upper(x x^T)] per point (N x F)."""
    X = np.asarray(X, dtype=np.float64)
    N, D = X.shape
    iu = np.triu_indices(D)
    outer = X[:, :, None] * X[:, None, :]
    return np.concatenate([np.ones((N, 1)), X, outer[:, iu[0], iu[1]]], axis=1)
