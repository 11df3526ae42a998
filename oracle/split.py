"""The split model of Sec. 2.1.2 (Fig. 3) -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline /
reference legs may import this module.  It shares no code with the CUDA
library; its Normal-Wishart pieces (posterior update, log rho, KL terms) are
those of ``oracle.py`` (the FP64 C oracle) applied to each 3-D block.

Each component k has a spatial Gaussian s | z=k ~ N(mu_s,k, Lambda_s,k^-1)
and a colour Gaussian c | z=k ~ N(mu_c,k, Lambda_c,k^-1), each with its own
Normal-Wishart prior and posterior, and one Dirichlet over the weights
(Fig. 3; Alg. 1 keeps separate spatial and colour statistics).  Hence
  log rho_nk = E[ln pi_k] + E[ln N(s_n | .)_k] + E[ln N(c_n | .)_k],
the statistics of each block are the count, its first moments and its own
second moments (the position-colour cross moments are not used), and the KL
of q against p is the Dirichlet term plus both blocks' Normal-Wishart terms.
Readings (each stated in the design notes): the hyper-parameters alpha0,
beta0, nu0 and the component means m0 are shared by the blocks unless
per-block beta0 / nu0 are given; the blocks' prior scales are the diagonal
blocks of the 6 x 6 W0; statistics keep the joint model's layout
[N, S1 (6), S2 upper (21)] so that the same E-step serves both models.

Pins: tests/test_split_pins.py (the K = 1 converged ELBO against the exact
log evidence of the two blocks, log rho against Monte Carlo expectations
drawn by scipy samplers, the ELBO of a small mixture against brute-force
enumeration of every hard assignment, the cross moments having no effect, the
ELBO's monotonicity and the count's conservation).
"""
from __future__ import annotations

import numpy as np

from . import oracle as O

D = 6
F = 28
BLOCKS = ((0, 3), (3, 6))   # spatial, colour coordinates


def _upper_index(i: int, j: int, d: int) -> int:
    """Position of (i, j), i <= j, in [N, S1 (d), S2 upper (row-major)]."""
    return 1 + d + i * d - i * (i - 1) // 2 + (j - i)


def block_stats(S, b: int) -> np.ndarray:
    """The block-b statistics (K x 10) of joint statistics S (K x 28)."""
    S = np.asarray(S, dtype=np.float64).reshape(-1, F)
    lo, hi = BLOCKS[b]
    d = hi - lo
    out = np.zeros((S.shape[0], 1 + d + d * (d + 1) // 2))
    out[:, 0] = S[:, 0]
    out[:, 1:1 + d] = S[:, 1 + lo:1 + hi]
    for i in range(d):
        for j in range(i, d):
            out[:, _upper_index(i, j, d)] = S[:, _upper_index(lo + i, lo + j, D)]
    return out


def block_priors(prior: dict, beta0_c=None, nu0_c=None):
    """The spatial and colour priors of a joint prior dict (m0 K x 6, W0 6 x 6)."""
    m0 = np.asarray(prior["m0"], dtype=np.float64)
    W0 = np.asarray(prior["W0"], dtype=np.float64)
    ps = {"alpha0": prior["alpha0"], "beta0": prior["beta0"], "nu0": prior["nu0"], "m0": m0[:, :3],
          "W0": W0[:3, :3]}
    pc = {"alpha0": prior["alpha0"], "beta0": prior["beta0"] if beta0_c is None else beta0_c,
          "nu0": prior["nu0"] if nu0_c is None else nu0_c, "m0": m0[:, 3:], "W0": W0[3:, 3:]}
    return ps, pc


def mstep(prior: dict, S, **kw):
    """update_from_statistics for both blocks: (q_s, q_c)."""
    ps, pc = block_priors(prior, **kw)
    return O.mstep(ps, block_stats(S, 0)), O.mstep(pc, block_stats(S, 1))


def e_ln_pi(alpha) -> np.ndarray:
    """E[ln pi_k] = psi(alpha_k) - psi(sum alpha)."""
    alpha = np.asarray(alpha, dtype=np.float64)
    return np.array([O.digamma(a) for a in alpha]) - O.digamma(float(alpha.sum()))


def log_rho(X, q_s: dict, q_c: dict) -> np.ndarray:
    """log rho_nk (N x K): each block's expected log-likelihood with E[ln pi]
    (as oracle.log_rho gives it), the E[ln pi] counted once."""
    X = np.asarray(X, dtype=np.float64)
    return O.log_rho(X[:, :3], q_s) + O.log_rho(X[:, 3:], q_c) - e_ln_pi(q_s["alpha"])[None, :]


def features(X) -> np.ndarray:
    """[1, x, upper(x x^T)] per point (N x 28)."""
    X = np.asarray(X, dtype=np.float64)
    iu = np.triu_indices(D)
    outer = X[:, :, None] * X[:, None, :]
    return np.concatenate([np.ones((X.shape[0], 1)), X, outer[:, iu[0], iu[1]]], axis=1)


def estep_stats(X, q_s: dict, q_c: dict):
    """(lse (N), dS (K x 28), R (N x K)) of one batch (compute_elbo_delta and
    Eq. 3's contraction R^T S_u)."""
    lr = log_rho(X, q_s, q_c)
    m = lr.max(axis=1, keepdims=True)
    lse = (m + np.log(np.exp(lr - m).sum(axis=1, keepdims=True)))[:, 0]
    R = np.exp(lr - lse[:, None])
    return lse, R.T @ features(X), R


def kl_total(q_s: dict, q_c: dict, p_s: dict, p_c: dict) -> float:
    """KL(q || p): the Dirichlet term and both blocks' Normal-Wishart terms."""
    K = q_s["alpha"].shape[0]
    kl = O.kl_dir(q_s["alpha"], p_s["alpha"])
    for k in range(K):
        kl += O.kl_nw(q_s, p_s, k) + O.kl_nw(q_c, p_c, k)
    return kl


def cavi_frame(X, prior: dict, S_past, n_iters: int, **kw):
    """One frame of Alg. 1 `fit` (the joint oracle's order): p = prior0 (+)
    S_past, q_0 = p; per iteration the E-step under q_t, elbo[t] =
    sum_n lse_n - KL(q_t || p), q_{t+1} = prior0 (+) (S_past + dS); then
    S_past += dS.  Returns (elbo trace, new S_past, lse, dS of the last
    iteration)."""
    X = np.asarray(X, dtype=np.float64)
    S_past = np.asarray(S_past, dtype=np.float64).reshape(-1, F)
    p_s, p_c = mstep(prior, S_past, **kw)
    q_s, q_c = p_s, p_c
    elbo = np.zeros(n_iters)
    lse, dS = np.zeros(X.shape[0]), np.zeros_like(S_past)
    for t in range(n_iters):
        lse, dS, _ = estep_stats(X, q_s, q_c)
        elbo[t] = lse.sum() - kl_total(q_s, q_c, p_s, p_c)
        q_s, q_c = mstep(prior, S_past + dS, **kw)
    return elbo, S_past + dS, lse, dS
