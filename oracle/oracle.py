"""FP64 CPU oracle of the VBGS CAVI update -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline /
reference legs may import this module.  It wraps ``vbgs_oracle.c`` (plain C,
FP64, OpenMP over points), which shares no code with the CUDA library.  See
that file's header for what each function computes and which part of the
paper it follows (Sec. 2.1.2 model, Alg. 1 `fit`, Eq. 3 fused contraction).

Pins: tests/test_oracle_pins.py checks these functions against closed forms
(K = 1 conjugate posterior and exact log evidence), brute-force enumeration,
Monte Carlo expectations drawn by library samplers, invariants and special
function values.  No function here is left "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "vbgs_oracle.c"
LIB = HERE / "libvbgs_oracle.so"

_DP = C.POINTER(C.c_double)


def build(force: bool = False) -> Path:
    """Compile the oracle (gcc, -O2, OpenMP, IEEE FP64: no fast-math)."""
    if not force and LIB.exists() and LIB.stat().st_mtime >= SRC.stat().st_mtime:
        return LIB
    tmp = LIB.with_suffix(".so.tmp")
    cmd = [os.environ.get("CC", "gcc"), "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           str(SRC), "-o", str(tmp), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(str(LIB))
        L.or_digamma.argtypes = [C.c_double]
        L.or_digamma.restype = C.c_double
        L.or_lmvgamma.argtypes = [C.c_int, C.c_double]
        L.or_lmvgamma.restype = C.c_double
        L.or_mstep.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, _DP, _DP, _DP,
                               _DP, _DP, _DP, _DP, _DP]
        L.or_mstep.restype = None
        L.or_log_rho.argtypes = [C.c_int, C.c_int, C.c_int, _DP, _DP, _DP, _DP, _DP, _DP, _DP]
        L.or_estep_stats.argtypes = [C.c_int, C.c_int, C.c_int, _DP, _DP, _DP, _DP, _DP, _DP, _DP, _DP, _DP]
        L.or_kl_nw.argtypes = [C.c_int, _DP, C.c_double, _DP, C.c_double, _DP, C.c_double, _DP, C.c_double]
        L.or_kl_nw.restype = C.c_double
        L.or_kl_dir.argtypes = [C.c_int, _DP, _DP]
        L.or_kl_dir.restype = C.c_double
        L.or_cavi_frame.argtypes = [C.c_int, C.c_int, C.c_int, _DP, C.c_double, C.c_double, C.c_double,
                                    _DP, _DP, _DP, C.c_int, _DP, _DP, _DP]
        L.or_elbo.argtypes = [C.c_int, C.c_int, C.c_int, _DP, C.c_double, C.c_double, C.c_double,
                              _DP, _DP, _DP, _DP, _DP]
        L.or_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _a(x, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    return a.reshape(shape) if shape is not None else a


def _p(a):
    return None if a is None else a.ctypes.data_as(_DP)


def F_of(D: int) -> int:
    return 1 + D + D * (D + 1) // 2


def num_threads() -> int:
    return int(lib().or_num_threads())


def digamma(x: float) -> float:
    return float(lib().or_digamma(float(x)))


def lmvgamma(D: int, a: float) -> float:
    return float(lib().or_lmvgamma(int(D), float(a)))


def mstep(prior: dict, S) -> dict:
    """update_from_statistics: posterior of every component from total stats S (K x F)."""
    m0 = _a(prior["m0"])
    K, D = m0.shape
    W0inv = np.linalg.inv(_a(prior["W0"]))
    W0inv = _a(0.5 * (W0inv + W0inv.T))
    S = _a(S, (K, F_of(D)))
    out = {"alpha": np.zeros(K), "beta": np.zeros(K), "nu": np.zeros(K), "m": np.zeros((K, D)),
           "Winv": np.zeros((K, D, D))}
    lib().or_mstep(K, D, prior["alpha0"], prior["beta0"], prior["nu0"], _p(m0), _p(W0inv), _p(S),
                   _p(out["alpha"]), _p(out["beta"]), _p(out["nu"]), _p(out["m"]), _p(out["Winv"]))
    return out


def log_rho(X, post: dict) -> np.ndarray:
    """log rho_nk of compute_elbo_delta for all pairs (N x K)."""
    X = _a(X)
    N, D = X.shape
    K = post["alpha"].shape[0]
    out = np.zeros((N, K))
    rc = lib().or_log_rho(N, K, D, _p(X), _p(_a(post["alpha"])), _p(_a(post["beta"])), _p(_a(post["nu"])),
                          _p(_a(post["m"])), _p(_a(post["Winv"])), _p(out))
    if rc:
        raise ArithmeticError(f"oracle: W^-1 of component {-rc - 1} not positive definite")
    return out


def estep_stats(X, post: dict, want_R: bool = False):
    """(lse (N), dS (K x F), R (N x K) or None) for one batch under posterior post."""
    X = _a(X)
    N, D = X.shape if X.size else (0, post["m"].shape[1])
    K = post["alpha"].shape[0]
    lse = np.zeros(max(N, 1))
    dS = np.zeros((K, F_of(D)))
    R = np.zeros((N, K)) if want_R else None
    rc = lib().or_estep_stats(N, K, D, _p(X) if N else None, _p(_a(post["alpha"])), _p(_a(post["beta"])),
                              _p(_a(post["nu"])), _p(_a(post["m"])), _p(_a(post["Winv"])), _p(lse), _p(dS), _p(R))
    if rc:
        raise ArithmeticError(f"oracle: W^-1 of component {-rc - 1} not positive definite")
    return lse[:N], dS, R


def kl_nw(q: dict, p: dict, k: int = 0) -> float:
    D = q["m"].shape[1]
    return float(lib().or_kl_nw(D, _p(_a(q["m"][k])), float(q["beta"][k]), _p(_a(q["Winv"][k])), float(q["nu"][k]),
                                _p(_a(p["m"][k])), float(p["beta"][k]), _p(_a(p["Winv"][k])), float(p["nu"][k])))


def kl_dir(alpha, alpha0) -> float:
    a = _a(alpha)
    return float(lib().or_kl_dir(a.shape[0], _p(a), _p(_a(alpha0))))


def cavi_frame(X, prior: dict, S_past, n_iters: int):
    """One frame of Alg. 1 fit.  Returns (elbo trace, new S_past, lse of the last
    E-step, Delta S of the last iteration)."""
    X = _a(X)
    m0 = _a(prior["m0"])
    K, D = m0.shape
    N = X.shape[0] if X.size else 0
    S = _a(S_past, (K, F_of(D))).copy()
    elbo = np.zeros(n_iters)
    lse = np.zeros(max(N, 1))
    dS = np.zeros((K, F_of(D)))
    rc = lib().or_cavi_frame(N, K, D, _p(X) if N else None, prior["alpha0"], prior["beta0"], prior["nu0"],
                             _p(m0), _p(_a(prior["W0"])), _p(S), int(n_iters), _p(elbo), _p(lse), _p(dS))
    if rc:
        raise ArithmeticError(f"oracle: cavi_frame failed ({rc})")
    return elbo, S, lse[:N], dS


def elbo(X, prior: dict, S_past, S_frame=None) -> float:
    """ELBO of prior0 (+) (S_past + S_frame) on X against prior0 (+) S_past."""
    X = _a(X)
    m0 = _a(prior["m0"])
    K, D = m0.shape
    N = X.shape[0] if X.size else 0
    out = np.zeros(1)
    rc = lib().or_elbo(N, K, D, _p(X) if N else None, prior["alpha0"], prior["beta0"], prior["nu0"], _p(m0),
                       _p(_a(prior["W0"])), _p(_a(S_past, (K, F_of(D)))),
                       None if S_frame is None else _p(_a(S_frame, (K, F_of(D)))), _p(out))
    if rc:
        raise ArithmeticError(f"oracle: elbo failed ({rc})")
    return float(out[0])


def relerr(y, yh, tau: float = 1e-30) -> float:
    """The paper's relative error (Eq. relerr): ||y_h - y||_2 / max(||y_h||_2, tau)."""
    y = np.asarray(y, dtype=np.float64).ravel()
    yh = np.asarray(yh, dtype=np.float64).ravel()
    return float(np.linalg.norm(yh - y) / max(np.linalg.norm(yh), tau))
