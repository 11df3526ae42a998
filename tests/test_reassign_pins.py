"""Pins of the oracle's reassign (Alg. 1, the step before fit) against
results other than itself (CPU only).

The sampling reading (n points drawn without replacement with probability
proportional to exp(-lse_n / tau), as the n largest Gumbel-perturbed keys) is
pinned by Monte Carlo with numpy's own Gumbel sampler against the softmax and
against the closed form of the two-of-three inclusion probabilities; the tie
rules and the component order by brute force over tuples; the
reinitialisation by the posterior of a component no data has reached.  A
wrong sign of the bias, a missing 1/tau, a reversed order or a write to the
wrong parameter fails one of them.
"""
from __future__ import annotations

import numpy as np
import pytest
from scipy.special import softmax

from oracle import oracle as O
from oracle import reassign as RA


def _prior(K, rng):
    A = rng.standard_normal((6, 6))
    return {"alpha0": 1.1, "beta0": 0.6, "nu0": 9.0, "m0": rng.standard_normal((K, 6)),
            "W0": A @ A.T / 6 + 0.5 * np.eye(6)}


def test_gumbel_top1_frequencies_are_softmax_of_minus_lse_over_tau():
    rng = np.random.default_rng(11)
    lse = np.array([0.3, -1.2, 2.0, 0.0, -0.4])
    tau, M = 0.7, 20000
    G = rng.gumbel(size=(M, lse.size))
    counts = np.zeros(lse.size)
    for row in G:
        counts[RA.pick_points(RA.point_keys(lse, row, tau), 1)[0]] += 1
    p = softmax(-lse / tau)
    se = np.sqrt(p * (1 - p) / M)
    assert np.all(np.abs(counts / M - p) < 5 * se + 1e-12), (counts / M, p)
    # the lowest lse is the most likely pick: the bias is toward low ELBO
    assert np.argmax(counts) == np.argmin(lse)


def test_gumbel_top2_of_3_excludes_each_item_with_the_plackett_luce_probability():
    rng = np.random.default_rng(12)
    lse = np.array([0.5, -0.3, 1.1])
    tau, M = 1.3, 20000
    w = np.exp(-lse / tau)
    W = w.sum()
    # P(i left out) = sum over the first pick j != i of w_j / W * w_k / (W - w_j), k the third item
    p_out = np.array([sum(w[j] / W * w[3 - i - j] / (W - w[j]) for j in range(3) if j != i) for i in range(3)])
    assert abs(p_out.sum() - 1.0) < 1e-12
    G = rng.gumbel(size=(M, 3))
    out = np.zeros(3)
    for row in G:
        picked = RA.pick_points(RA.point_keys(lse, row, tau), 2)
        out[3 - picked[0] - picked[1]] += 1
    se = np.sqrt(p_out * (1 - p_out) / M)
    assert np.all(np.abs(out / M - p_out) < 5 * se), (out / M, p_out)


def test_noiseless_keys_pick_the_lowest_lse_ties_to_the_lower_index():
    lse = np.array([1.0, 0.5, 0.5, 2.0, 0.5, -1.0])
    picked = RA.pick_points(RA.point_keys(lse, np.zeros(6), 1.0), 4)
    assert picked.tolist() == [5, 1, 2, 4]
    # a scale 1/tau changes nothing without noise
    assert RA.pick_points(RA.point_keys(lse, np.zeros(6), 0.25), 4).tolist() == [5, 1, 2, 4]


def test_component_order_matches_brute_force_over_tuples():
    rng = np.random.default_rng(13)
    K = 60
    counts = rng.choice([0.0, 0.0, 0.0, 1.5, 2.0, 7.25], size=K)
    v = rng.choice([0.1, 0.2, 0.3], size=K)
    for n in (1, 7, 25, K):
        want = sorted(range(K), key=lambda k: (counts[k], v[k], k))[:n]
        assert RA.pick_components(counts, n, v).tolist() == want
        want0 = sorted(range(K), key=lambda k: (counts[k], k))[:n]
        assert RA.pick_components(counts, n, None).tolist() == want0
    # -0.0 and +0.0 tie
    c = np.array([0.0, -0.0, 0.0])
    assert RA.pick_components(c, 3, None).tolist() == [0, 1, 2]


def test_reassign_moves_only_the_prior_means_of_least_used_components():
    rng = np.random.default_rng(14)
    K, N = 12, 40
    prior = _prior(K, rng)
    X = rng.standard_normal((N, 6))
    # statistics: components 0..5 visited, 6..11 never
    _, S, _ = O.estep_stats(X, O.mstep(prior, np.zeros((K, 28))))
    S[6:] = 0.0
    assert np.all(S[:6, 0] > 0)
    g = rng.gumbel(size=N)
    pts, comps, m0_new, lse = RA.reassign(X, prior, S, 4, g, tau=1.0)
    assert set(comps.tolist()) <= set(range(6, 12))                # least used: the unvisited ones
    assert np.array_equal(m0_new[comps], X[pts])
    keep = np.setdiff1d(np.arange(K), comps)
    assert np.array_equal(m0_new[keep], prior["m0"][keep])
    # the posterior of a reinitialised unvisited component is the prior around the sampled point
    prior_new = dict(prior, m0=m0_new)
    post = O.mstep(prior_new, S)
    W0inv = np.linalg.inv(prior["W0"])
    for i, k in enumerate(comps):
        assert np.allclose(post["m"][k], X[pts[i]], rtol=0, atol=1e-14)
        assert np.allclose(post["Winv"][k], W0inv, rtol=1e-12, atol=1e-12)
        assert post["alpha"][k] == prior["alpha0"] and post["nu"][k] == prior["nu0"]
    # the lse ranked on is the per-point ELBO term of the unchanged posterior
    assert np.array_equal(lse, O.estep_stats(X, O.mstep(prior, S))[0])


def test_reassign_is_invariant_under_a_permutation_of_the_points():
    rng = np.random.default_rng(15)
    K, N = 10, 50
    prior = _prior(K, rng)
    X = rng.standard_normal((N, 6))
    S = np.zeros((K, 28))
    S[:, 0] = rng.choice([0.0, 1.0, 3.0], size=K)
    g = rng.gumbel(size=N)
    v = rng.random(K)
    pts, comps, m0, _ = RA.reassign(X, prior, S, 5, g, tau=2.0, comp_key=v)
    perm = rng.permutation(N)
    pts2, comps2, m02, _ = RA.reassign(X[perm], prior, S, 5, g[perm], tau=2.0, comp_key=v)
    assert np.array_equal(perm[pts2], pts)
    assert np.array_equal(comps2, comps) and np.array_equal(m02, m0)


def test_reassign_argument_errors():
    rng = np.random.default_rng(16)
    prior = _prior(3, rng)
    X = rng.standard_normal((5, 6))
    with pytest.raises(ValueError):
        RA.reassign(X, prior, np.zeros((3, 28)), 4, np.zeros(5))
    pts, comps, m0, _ = RA.reassign(X, prior, np.zeros((3, 28)), 0, np.zeros(5))
    assert pts.size == 0 and comps.size == 0 and np.array_equal(m0, prior["m0"])
