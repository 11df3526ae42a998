"""reassign of Alg. 1 (the step before fit in every frame; Sec. 2.1.2) --
TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline /
reference legs may import this module.  It shares no code with the CUDA
library; the per-point ELBO terms come from ``oracle.py`` (the FP64 C oracle).

Alg. 1 and the text after it: evaluate the per-point ELBO of the frame,
sample n points biased toward low ELBO, pick n least-used components and
reinitialise them by setting their spatial and colour means (the prior means
m0 of the initialisation model; nothing else changes) to the sampled points.
Readings where the paper is silent (each stated in the design notes):

* per-point ELBO = lse_n, the log normaliser of point n's responsibilities
  under the current posterior prior0 (+) S (the part of the ELBO that depends
  on the point; the KL terms are shared by all points);
* "biased to low ELBO" = n distinct points drawn with probability
  proportional to exp(-lse_n / tau): the n largest keys g_n - lse_n / tau,
  g_n standard Gumbel variates supplied by the caller (the Gumbel-top-k
  construction of sampling without replacement: Vieira 2014; Kool, van Hoof
  and Welling 2019), ties to the lower index;
* "least-used" = smallest count N_k of S; ties by a caller-supplied key v_k,
  then by the lower index.  Components no data has reached (N_k = 0) all tie,
  so a random v picks among them at random, which is the text's "randomly
  among those not yet updated";
* the i-th sampled point (by key rank) becomes the mean of the i-th picked
  component.

Pins: tests/test_reassign_pins.py (Gumbel-max frequencies against
softmax(-lse / tau) by Monte Carlo, the noiseless case against the n lowest
lse, the component order against brute-force sorting of (N_k, v_k, k), the
reinitialised posterior mean of an unvisited component against the sampled
point, and invariance under a permutation of the points); lse_n is
``oracle.estep_stats``, pinned in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def point_keys(lse, gumbel, tau: float) -> np.ndarray:
    """g_n - lse_n / tau (the product rounded, then the difference)."""
    lse = np.asarray(lse, dtype=np.float64)
    g = np.asarray(gumbel, dtype=np.float64)
    return g - lse * (1.0 / tau)


def pick_points(keys, n: int) -> np.ndarray:
    """Indices of the n largest keys, largest first, ties to the lower index."""
    keys = np.asarray(keys, dtype=np.float64)
    order = np.lexsort((np.arange(keys.size), -keys))   # primary -key, then index
    return order[:n].astype(np.int64)


def pick_components(counts, n: int, comp_key=None) -> np.ndarray:
    """Indices of the n least-used components: ascending N_k, then v_k, then k."""
    counts = np.asarray(counts, dtype=np.float64)
    K = counts.size
    v = np.zeros(K) if comp_key is None else np.asarray(comp_key, dtype=np.float64)
    order = np.lexsort((np.arange(K), v, counts))       # primary N_k, then v, then index
    return order[:n].astype(np.int64)


def lse_of(X, prior: dict, S) -> np.ndarray:
    """Per-point ELBO term lse_n under prior0 (+) S (update_from_statistics,
    then compute_elbo_delta of Alg. 1)."""
    post = O.mstep(prior, S)
    lse, _, _ = O.estep_stats(X, post)
    return lse


def reassign(X, prior: dict, S, n: int, gumbel, tau: float = 1.0, comp_key=None):
    """Returns (picked points, picked components, new m0 (K x 6), lse)."""
    X = np.asarray(X, dtype=np.float64)
    m0 = np.array(prior["m0"], dtype=np.float64)
    K = m0.shape[0]
    if not 0 <= n <= min(X.shape[0], K):
        raise ValueError("need 0 <= n <= min(N, K)")
    S = np.asarray(S, dtype=np.float64).reshape(K, -1)
    lse = lse_of(X, prior, S) if X.shape[0] else np.zeros(0)
    pts = pick_points(point_keys(lse, gumbel, tau), n)
    comps = pick_components(S[:, 0], n, comp_key)
    m0[comps] = X[pts]
    return pts, comps, m0, lse
