"""Planted mistakes in the oracle (CPU only).

Each case copies an oracle source, plants one plausible mistake in it (a
dropped term, a wrong sign, an index off by one, a forgotten statistic, a
reversed order) and loads the copy in place of the original: the C oracle
compiled into a temporary directory, a Python oracle module executed as a
fresh module.  At least one pin of that part of the oracle must then fail:
the pins fix the oracle's arithmetic against results other than itself, so a
mistake of this kind cannot pass them.  Nothing here touches a GPU.
"""
from __future__ import annotations

import ctypes
import importlib
import inspect
import os
import subprocess
import types
from pathlib import Path

import pytest

from oracle import oracle as O
from tests import test_oracle_pins as PINS
from tests import test_reassign_pins as PINS_RA
from tests import test_render_pins as PINS_RD
from tests import test_split_pins as PINS_SP

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


# Python oracle modules: (module, what is wrong, exact text, planted replacement)
PY_MUTANTS = [
    ("reassign", "keys biased toward high lse", "return g - lse * (1.0 / tau)", "return g + lse * (1.0 / tau)"),
    ("reassign", "keys scaled by tau instead of 1 / tau", "return g - lse * (1.0 / tau)", "return g - lse * tau"),
    ("reassign", "the n smallest keys picked", "order = np.lexsort((np.arange(keys.size), -keys))",
     "order = np.lexsort((np.arange(keys.size), keys))"),
    ("reassign", "components ordered by the tie key before the count",
     "order = np.lexsort((np.arange(K), v, counts))", "order = np.lexsort((np.arange(K), counts, v))"),
    ("reassign", "points paired with components in reverse", "m0[comps] = X[pts]", "m0[comps] = X[pts[::-1]]"),
    ("reassign", "the whole mean row but the colour replaced", "m0[comps] = X[pts]",
     "m0[comps, :3] = X[pts, :3]"),
    ("render", "expected covariance over nu - d", "/ (nu - d - 1.0)[:, None, None]", "/ (nu - d)[:, None, None]"),
    ("render", "Jacobian entry of the wrong sign", "J[:, 0, 2] = -f * xc[:, 0] / zs ** 2",
     "J[:, 0, 2] = f * xc[:, 0] / zs ** 2"),
    ("render", "screen covariance without the low-pass", "+ LOW_PASS * np.eye(2)[None, :, :]", ""),
    ("render", "back-to-front order", "order = keep[np.lexsort((keep, z[keep]))]",
     "order = keep[np.lexsort((keep, -z[keep]))]"),
    ("render", "colour added without the transmittance", "out += (T * a)[:, None] * colour[k][None, :]",
     "out += a[:, None] * colour[k][None, :]"),
    ("render", "splats behind the camera kept", "keep = np.flatnonzero(z > NEAR)", "keep = np.arange(z.size)"),
    ("render", "pixel corners for pixel centres", "np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)",
     "np.meshgrid(np.arange(W), np.arange(H))"),
    ("render", "components without data drawn", ">= MIN_COUNT)", "> 0.0)"),
    ("render", "PSNR with 20 log10", "10.0 * np.log10(255.0 ** 2 / mse)", "20.0 * np.log10(255.0 ** 2 / mse)"),
    ("split", "E[ln pi_k] counted twice", " - e_ln_pi(q_s[\"alpha\"])[None, :]", ""),
    ("split", "colour second moments read from the spatial block",
     "S[:, _upper_index(lo + i, lo + j, D)]", "S[:, _upper_index(i, j, D)]"),
    ("split", "colour prior scale from the spatial block", "\"W0\": W0[3:, 3:]", "\"W0\": W0[:3, :3]"),
    ("split", "KL without the colour block", "kl += O.kl_nw(q_s, p_s, k) + O.kl_nw(q_c, p_c, k)",
     "kl += O.kl_nw(q_s, p_s, k)"),
    ("split", "responsibilities against the row maximum", "R = np.exp(lr - lse[:, None])", "R = np.exp(lr - m)"),
    ("split", "stream that forgets S_past", "return elbo, S_past + dS, lse, dS", "return elbo, dS, lse, dS"),
    ("mlp", "softmax cross-entropy gradient of the wrong sign", "dz = (np.exp(log_softmax(z)) - q) / B",
     "dz = (q - np.exp(log_softmax(z))) / B"),
    ("mlp", "gradient without the 1 / B of the mean", "dz = (np.exp(log_softmax(z)) - q) / B",
     "dz = np.exp(log_softmax(z)) - q"),
    ("mlp", "ReLU mask of the wrong layer", "dh2 = (dz @ W3) * (h2 > 0)", "dh2 = (dz @ W3) * (h1 > 0)"),
    ("mlp", "first bias gradient from the second layer", "gW1, gb1 = dh1.T @ x, dh1.sum(0)",
     "gW1, gb1 = dh1.T @ x, dh2.sum(0)"),
    ("mlp", "loss summed instead of averaged", ".sum() / x.shape[0])", ".sum())"),
    ("mlp", "top-4 ties to the higher index", "idx = np.argsort(-np.asarray(z), axis=1, kind=\"stable\")",
     "idx = np.argsort(np.asarray(z), axis=1, kind=\"stable\")[:, ::-1]"),
]
PIN_MODULES = {"reassign": (PINS_RA, "RA"), "render": (PINS_RD, "RD"), "split": (PINS_SP, "SP"), "mlp": (None, None)}
# the MLP pins import oracle.mlp inside each function
MLP_PINS = (PINS.test_mlp_gradient_matches_central_differences, PINS.test_mlp_loss_closed_forms,
            PINS.test_top4_and_nearest_centroid_tie_rules)


def use_mutant(monkeypatch, module, mod):
    """Put the mutant where the module's pins look it up; returns those pins."""
    pins_module, name = PIN_MODULES[module]
    if pins_module is None:
        import oracle as pkg
        import sys
        monkeypatch.setitem(sys.modules, f"oracle.{module}", mod)
        monkeypatch.setattr(pkg, module, mod)
        return list(MLP_PINS)
    monkeypatch.setattr(pins_module, name, mod)
    return module_pins(pins_module)


def load_py_mutant(module, old, new):
    orig = importlib.import_module(f"oracle.{module}")
    path = Path(orig.__file__)
    src = path.read_text()
    assert src.count(old) == 1, f"oracle/{module}.py no longer holds the text to mutate: {old!r}"
    mod = types.ModuleType(f"oracle.{module}")
    mod.__file__, mod.__package__ = str(path), "oracle"
    exec(compile(src.replace(old, new), str(path), "exec"), mod.__dict__)
    return mod


def module_pins(pins_module):
    return [f for name, f in sorted(vars(pins_module).items())
            if name.startswith("test_") and inspect.isfunction(f) and not inspect.signature(f).parameters]


@pytest.mark.parametrize("module,what,old,new", PY_MUTANTS, ids=[f"{m[0]}: {m[1]}" for m in PY_MUTANTS])
def test_a_pin_fails_on_a_planted_mistake_in_a_python_module(monkeypatch, module, what, old, new):
    for pin in use_mutant(monkeypatch, module, load_py_mutant(module, old, new)):
        try:
            pin()
        except Exception:
            return
    pytest.fail(f"every pin of oracle/{module}.py passes with the planted mistake: {what}")


@pytest.mark.parametrize("module", sorted(PIN_MODULES))
def test_an_unmutated_python_module_passes_its_pins(monkeypatch, module):
    src = Path(importlib.import_module(f"oracle.{module}").__file__).read_text()
    line = next(l for l in src.splitlines() if l.strip() and not l.startswith(("#", '"', "from", "import", " ")))
    for pin in use_mutant(monkeypatch, module, load_py_mutant(module, line, line)):
        pin()
