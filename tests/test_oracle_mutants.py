"""Planted mistakes in the FP64 oracle (CPU only).

Each case copies the oracle's C source, plants one plausible mistake in it
(a dropped term, a wrong sign, an index off by one, a forgotten statistic),
compiles the copy into a temporary directory and loads it in place of the
oracle's library.  At least one pin of test_oracle_pins must then fail: the
pins fix the oracle's arithmetic against results other than itself, so a
mistake of this kind cannot pass them.  Nothing here touches a GPU.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import pytest

from oracle import oracle as O
from tests import test_oracle_pins as PINS

# (what is wrong, exact text of the oracle, planted replacement)
MUTANTS = [
    ("log rho without the D / (2 beta_k) term",
     "- 0.5 * D * log(2.0 * OR_PI) - 0.5 * D / beta[k];", "- 0.5 * D * log(2.0 * OR_PI);"),
    ("E[ln|Lambda_k|] without D ln 2",
     "or_mvdigamma(D, 0.5 * nu[k]) + D * log(2.0) - logdet_Winv", "or_mvdigamma(D, 0.5 * nu[k]) - logdet_Winv"),
    ("E[ln|Lambda_k|] with ln|W_k| of the wrong sign",
     "+ D * log(2.0) - logdet_Winv", "+ D * log(2.0) + logdet_Winv"),
    ("E[ln pi_k] without psi(sum alpha)",
     "cst[k] = or_digamma(alpha[k]) - psi_sum + 0.5 * elogdet", "cst[k] = or_digamma(alpha[k]) + 0.5 * elogdet"),
    ("quadratic form without nu_k",
     "return cstk - 0.5 * nuk * q;", "return cstk - 0.5 * q;"),
    ("log-sum-exp without the maximum added back",
     "double l = mx + log(s);", "double l = log(s);"),
    ("second-moment feature x_i x_i in place of x_i x_j",
     "phi[u++] = x[i] * x[j];", "phi[u++] = x[i] * x[i];"),
    ("posterior alpha without the count",
     "alpha[k] = alpha0 + Nk;", "alpha[k] = alpha0;"),
    ("posterior nu off by one",
     "nu[k] = nu0 + Nk;", "nu[k] = nu0 + Nk + 1.0;"),
    ("posterior mean without beta0 weighting m0",
     "(beta0 * m0[(size_t)k * D + i] + s[1 + i]) / beta[k]", "(m0[(size_t)k * D + i] + s[1 + i]) / beta[k]"),
    ("posterior W^-1 with + beta m m^T",
     "- beta[k] * m[(size_t)k * D + i] * m[(size_t)k * D + j];",
     "+ beta[k] * m[(size_t)k * D + i] * m[(size_t)k * D + j];"),
    ("posterior W^-1 reading the statistic before the right one",
     "double v = W0inv[i * D + j] + s[u]", "double v = W0inv[i * D + j] + s[u - 1]"),
    ("KL(NW) with the (nu - nu0)/2 psi_D term of the wrong sign",
     "kl += 0.5 * (nq - np) * or_mvdigamma", "kl += -0.5 * (nq - np) * or_mvdigamma"),
    ("KL(NW) without the trace term",
     "- 0.5 * nq * D + 0.5 * nq * tr", "- 0.5 * nq * D"),
    ("KL(NW) Mahalanobis term without nu",
     "bp * nq * maha", "bp * maha"),
    ("KL(Dirichlet) with psi(sum alpha) of the wrong sign",
     "(or_digamma(a[k]) - psi_as)", "(or_digamma(a[k]) + psi_as)"),
    ("digamma with +1/(2x)",
     "return acc + log(x) - 0.5 / x - series;", "return acc + log(x) + 0.5 / x - series;"),
    ("ln Gamma_D with the pi constant doubled",
     "0.25 * D * (D - 1) * log(OR_PI)", "0.5 * D * (D - 1) * log(OR_PI)"),
    # mistakes that leave one component unchanged, so that K = 1 pins cannot see them
    ("responsibilities not normalised by lse_n",
     "double r = exp(lr[k] - l);", "double r = exp(lr[k] - mx);"),
    ("psi(sum alpha) from the last component's alpha only",
     "for (int k = 0; k < K; k++) asum += alpha[k];", "for (int k = 0; k < K; k++) asum = alpha[k];"),
    ("posterior of component k from the statistics of component K - 1 - k",
     "const double *s = S + (size_t)k * F;", "const double *s = S + (size_t)(K - 1 - k) * F;"),
    ("stream that replaces S_past by the frame's statistics",
     "for (size_t i = 0; i < (size_t)K * F; i++) S_past[i] += dS[i];",
     "for (size_t i = 0; i < (size_t)K * F; i++) S_past[i] = dS[i];"),
]

# the entry points the pins reach through oracle.lib()
ENTRY = ("or_digamma", "or_lmvgamma", "or_mstep", "or_log_rho", "or_estep_stats", "or_kl_nw", "or_kl_dir",
         "or_cavi_frame", "or_elbo", "or_num_threads")


def pins():
    """The pins, cheapest first (the two Monte Carlo pins last)."""
    return [
        PINS.test_digamma_golden_values,
        PINS.test_digamma_and_mvgamma_vs_scipy,
        lambda: PINS.test_k1_posterior_and_elbo_equal_exact_evidence(7),
        PINS.test_streaming_k1_equals_batch_posterior,
        PINS.test_hard_assignment_mstep_is_per_cluster_conjugate_update,
        PINS.test_responsibilities_are_softmax_of_log_rho_and_stats_are_eq3,
        PINS.test_bruteforce_evidence_k1_equality,
        PINS.test_bruteforce_evidence_bounds_every_elbo,
        PINS.test_kl_dirichlet_matches_monte_carlo,
        PINS.test_elbo_non_decreasing_on_mixture_workload,
        PINS.test_log_rho_matches_monte_carlo_expectation,
        PINS.test_kl_nw_matches_monte_carlo_and_vanishes_at_equality,
    ]


def load_mutant(tmp_path, old, new):
    src = O.SRC.read_text()
    assert src.count(old) == 1, f"the oracle no longer holds the text to mutate: {old!r}"
    c = tmp_path / "mutant.c"
    c.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run([os.environ.get("CC", "gcc"), "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", str(c),
                    "-o", str(so), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    ref = O.lib()
    for name in ENTRY:
        f, g = getattr(lib, name), getattr(ref, name)
        f.argtypes, f.restype = g.argtypes, g.restype
    return lib


@pytest.mark.parametrize("what,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_a_pin_fails_on_the_planted_mistake(tmp_path, monkeypatch, what, old, new):
    monkeypatch.setattr(O, "_lib", load_mutant(tmp_path, old, new))
    for pin in pins():
        try:
            pin()
        except Exception:   # an assertion, or a non-PD posterior the mistake caused
            return
    pytest.fail(f"every pin passes with the planted mistake: {what}")


def test_the_unmutated_copy_passes_every_pin(tmp_path, monkeypatch):
    """The harness itself: a copy compiled the same way, with nothing planted."""
    monkeypatch.setattr(O, "_lib", load_mutant(tmp_path, "double l = mx + log(s);", "double l = mx + log(s);"))
    for pin in pins():
        pin()
