"""Thin ctypes binding of the C ABI in include/vbgs.h.

Argument marshalling only: every step of the CAVI update runs in the CUDA
kernels of ``libvbgs.so``.  The functions keep the C names (``vbgs_init``,
``vbgs_update``, ``vbgs_elbo``, ``vbgs_get_posterior``, ...); the ``Model``
class wraps a context for convenience.  Arrays may be numpy arrays (host) or
torch tensors (host or CUDA); torch is used only for device memory and the
current stream.  Importing this module fails loudly if the library is
missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "libvbgs.so"

VBGS_OK = 0
VBGS_EINVAL = -1
VBGS_ENOMEM = -2
VBGS_ECUDA = -3
VBGS_ENUMERIC = -4
VBGS_ETIMEOUT = -5
VBGS_ECHECK = -6
VBGS_EIO = -7

VBGS_FP64 = 0
VBGS_FP16X3 = 1
VBGS_BF16X3 = 2
VBGS_FP32 = 3
PRECISIONS = {"fp64": VBGS_FP64, "fp16x3": VBGS_FP16X3, "bf16x3": VBGS_BF16X3, "fp32": VBGS_FP32}
VBGS_FLAG_NO_REORDER = 1
VBGS_FLAG_NO_SKIP = 2
VBGS_FLAG_PLAIN = VBGS_FLAG_NO_REORDER | VBGS_FLAG_NO_SKIP
VBGS_FLAG_PROPOSAL = 4
VBGS_FLAG_SPLIT = 8
PROP_CLUSTERS = 1024
PROP_NPARAM = 128 * 6 + 128 + 128 * 128 + 128 + 1024 * 128 + 1024
PROP_REPORT = ["cand_pairs", "fallback", "audit", "audit_max_missed", "audit_mean_missed", "frame_exact",
               "train_loss", "frames_trained", "exact_pairs", "points", "added_clusters"]

D = 6
F = 28

# Every symbol include/vbgs.h declares (checked by the ABI test).
EXPORTS = [
    "vbgs_init", "vbgs_update", "vbgs_elbo", "vbgs_get_posterior", "vbgs_get_stats",
    "vbgs_set_stats", "vbgs_get_frame_stats", "vbgs_get_lse", "vbgs_last_launch_count",
    "vbgs_profile_enable", "vbgs_profile_read", "vbgs_profile_pairs", "vbgs_profile_name", "vbgs_probe_peaks",
    "vbgs_estep_noalloc", "vbgs_update_batched", "vbgs_autotune", "vbgs_get_tuning", "vbgs_set_tuning",
    "vbgs_proposal_report", "vbgs_proposal_config", "vbgs_proposal_weights", "vbgs_proposal_grad",
    "vbgs_proposal_clusters",
    "vbgs_proposal_bounds", "vbgs_kmeans", "vbgs_reassign", "vbgs_save_state", "vbgs_load_state",
    "vbgs_check_frame", "vbgs_set_wait_limit", "vbgs_render", "vbgs_profile_replay", "vbgs_set_precision_knobs",
    "vbgs_get_precision_knobs", "vbgs_last_error", "vbgs_destroy",
]
KNOBS = ["P1_PHI_LO", "P1_C_LO", "P2_PHI_LO", "P2_C_LO", "P2_P_LO", "P2_S_LO"]   # bit i: leave that lo term out
NOALLOC_SCRATCH_BYTES = 24 * 1024 * 1024
PROF_COUNT = 8
PROF_NAMES = ["pass1", "merge", "pass2", "reduce", "mstep", "misc", "plan", "kl"]


class VbgsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"vbgs error {code}: {msg}")
        self.code = code


class vbgs_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("flags", C.c_int), ("cuda_stream", C.c_void_p),
                ("checks", C.c_int), ("autotune_cache", C.c_char_p), ("seed", C.c_uint64)]


class vbgs_prior(C.Structure):
    _fields_ = [("alpha0", C.c_double), ("beta0", C.c_double), ("nu0", C.c_double),
                ("m0", C.POINTER(C.c_double)), ("W0", C.POINTER(C.c_double))]


_DP = C.POINTER(C.c_double)


def load_library(path: Path | str = LIB_PATH) -> C.CDLL:
    path = Path(path)
    if not path.exists():
        raise ImportError(f"{path} is missing: run __graft_entry__.build() (no CPU fallback exists)")
    lib = C.CDLL(str(path))
    lib.vbgs_init.argtypes = [C.POINTER(C.c_void_p), C.POINTER(vbgs_prior), C.c_int, C.c_int,
                              C.POINTER(vbgs_options)]
    lib.vbgs_update.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, _DP]
    lib.vbgs_elbo.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, _DP, _DP]
    lib.vbgs_reassign.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_double, _DP, _DP,
                                  C.POINTER(C.c_int64), C.POINTER(C.c_int)]
    lib.vbgs_get_posterior.argtypes = [C.c_void_p, _DP, _DP, _DP, _DP, _DP]
    lib.vbgs_get_stats.argtypes = [C.c_void_p, _DP]
    lib.vbgs_set_stats.argtypes = [C.c_void_p, _DP]
    lib.vbgs_get_frame_stats.argtypes = [C.c_void_p, _DP]
    lib.vbgs_get_lse.argtypes = [C.c_void_p, _DP, C.c_int64]
    lib.vbgs_last_launch_count.argtypes = [C.c_void_p]
    lib.vbgs_last_launch_count.restype = C.c_int64
    lib.vbgs_last_error.argtypes = [C.c_void_p]
    lib.vbgs_last_error.restype = C.c_char_p
    lib.vbgs_destroy.argtypes = [C.c_void_p]
    lib.vbgs_destroy.restype = None
    lib.vbgs_profile_enable.argtypes = [C.c_void_p, C.c_int]
    lib.vbgs_profile_read.argtypes = [C.c_void_p, _DP, C.POINTER(C.c_int64), C.c_int]
    lib.vbgs_profile_pairs.argtypes = [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    lib.vbgs_profile_name.argtypes = [C.c_int]
    lib.vbgs_profile_name.restype = C.c_char_p
    lib.vbgs_probe_peaks.argtypes = [C.c_int, _DP]
    lib.vbgs_estep_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    lib.vbgs_update_batched.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p),
                                        C.POINTER(C.c_int64), C.c_int, _DP]
    lib.vbgs_autotune.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_char_p]
    lib.vbgs_get_tuning.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.vbgs_set_tuning.argtypes = [C.c_void_p, C.c_int, C.c_int]
    _FP = C.POINTER(C.c_float)
    lib.vbgs_proposal_report.argtypes = [C.c_void_p, _DP]
    lib.vbgs_proposal_config.argtypes = [C.c_void_p, C.c_int, C.c_double]
    lib.vbgs_proposal_weights.argtypes = [C.c_void_p, _FP, _FP]
    lib.vbgs_proposal_grad.argtypes = [C.c_void_p, _FP, _FP, C.c_int, _FP, _FP, C.POINTER(C.c_int)]
    lib.vbgs_proposal_clusters.argtypes = [C.c_void_p, _FP, C.POINTER(C.c_int)]
    lib.vbgs_proposal_bounds.argtypes = [C.c_void_p, _DP, C.c_int64, _FP, C.POINTER(C.c_int)]
    lib.vbgs_kmeans.argtypes = [_FP, C.c_int, _FP, C.c_int, C.POINTER(C.c_int)]
    lib.vbgs_save_state.argtypes = [C.c_void_p, C.c_char_p]
    lib.vbgs_load_state.argtypes = [C.POINTER(C.c_void_p), C.c_char_p, C.POINTER(vbgs_options)]
    lib.vbgs_check_frame.argtypes = [_DP, C.c_int, _DP, C.c_int64, _DP, C.c_double, C.POINTER(C.c_int)]
    lib.vbgs_set_wait_limit.argtypes = [C.c_longlong]
    lib.vbgs_render.argtypes = [C.c_void_p, _DP, C.c_int, C.c_int, _FP, _FP, _DP, _DP]
    lib.vbgs_profile_replay.argtypes = [C.c_void_p, C.c_int, _DP, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    lib.vbgs_set_precision_knobs.argtypes = [C.c_void_p, C.c_uint]
    lib.vbgs_get_precision_knobs.argtypes = [C.c_void_p]
    lib.vbgs_get_precision_knobs.restype = C.c_uint
    return lib


_lib: C.CDLL | None = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def _check(rc: int, ctx=None) -> None:
    if rc != VBGS_OK:
        raise VbgsError(rc, lib().vbgs_last_error(ctx).decode(errors="replace"))


def _host_f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None and a.shape != shape:
        a = a.reshape(shape)
    return a


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _points_ptr(points):
    """(pointer, N, keepalive) for an N x 6 float64 array on host or device."""
    try:
        import torch
        if isinstance(points, torch.Tensor):
            if points.dtype != torch.float64 or points.dim() != 2 or points.shape[1] != D:
                raise ValueError("points must be an N x 6 float64 tensor")
            t = points.contiguous()
            return C.c_void_p(t.data_ptr() if t.numel() else None), t.shape[0], t
    except ImportError:
        pass
    a = _host_f64(points)
    if a.ndim != 2 or a.shape[1] != D:
        raise ValueError("points must be N x 6")
    return C.c_void_p(a.ctypes.data if a.size else None), a.shape[0], a


# ---- C-named functions ------------------------------------------------------

def _options(precision: int = VBGS_FP64, flags: int = 0, cuda_stream: int | None = None, checks: bool = False,
             autotune_cache: str | None = None, seed: int = 0) -> vbgs_options:
    return vbgs_options(int(precision), int(flags), C.c_void_p(cuda_stream or None), int(bool(checks)),
                        autotune_cache.encode() if autotune_cache else None, int(seed))


def vbgs_init(alpha0: float, beta0: float, nu0: float, m0, W0, precision: int = VBGS_FP64,
              cuda_stream: int | None = None, flags: int = 0, checks: bool = False,
              autotune_cache: str | None = None, seed: int = 0):
    m0a = _host_f64(m0)
    K = m0a.shape[0]
    W0a = _host_f64(W0, (D, D))
    pr = vbgs_prior(alpha0, beta0, nu0, _dp(m0a), _dp(W0a))
    opt = _options(precision, flags, cuda_stream, checks, autotune_cache, seed)
    ctx = C.c_void_p()
    _check(lib().vbgs_init(C.byref(ctx), C.byref(pr), K, m0a.shape[1], C.byref(opt)), None)
    return ctx


def vbgs_save_state(ctx, path: str) -> None:
    _check(lib().vbgs_save_state(ctx, str(path).encode()), ctx)


def vbgs_load_state(path: str, cuda_stream: int | None = None, checks: bool = False,
                    autotune_cache: str | None = None):
    opt = _options(cuda_stream=cuda_stream, checks=checks, autotune_cache=autotune_cache)
    ctx = C.c_void_p()
    _check(lib().vbgs_load_state(C.byref(ctx), str(path).encode(), C.byref(opt)), None)
    return ctx


def vbgs_check_frame(dS, points, lse=None, tol: float = 1e-9) -> bool:
    """The frame consistency check of options.checks on host arrays."""
    S = _host_f64(dS)
    X = _host_f64(points)
    if S.ndim != 2 or S.shape[1] != F or X.ndim != 2 or X.shape[1] != D:
        raise ValueError("dS must be K x 28 and points N x 6")
    lp = None
    if lse is not None:
        la = _host_f64(lse).ravel()
        if la.size != X.shape[0]:
            raise ValueError("lse needs one value per point")
        lp = _dp(la)
    ok = C.c_int(0)
    _check(lib().vbgs_check_frame(_dp(S), S.shape[0], _dp(X) if X.size else None, X.shape[0], lp, float(tol),
                                  C.byref(ok)), None)
    return bool(ok.value)


def vbgs_update(ctx, points, n_iters: int) -> np.ndarray:
    ptr, N, keep = _points_ptr(points)
    trace = np.zeros(max(n_iters, 1), dtype=np.float64)
    _check(lib().vbgs_update(ctx, ptr, N, n_iters, _dp(trace)), ctx)
    del keep
    return trace[:n_iters]


def vbgs_elbo(ctx, points, want_lse: bool = False):
    ptr, N, keep = _points_ptr(points)
    out = np.zeros(1)
    lse = np.zeros(max(N, 1)) if want_lse else None
    _check(lib().vbgs_elbo(ctx, ptr, N, _dp(out), _dp(lse) if want_lse else None), ctx)
    del keep
    return (float(out[0]), lse[:N]) if want_lse else float(out[0])


def vbgs_reassign(ctx, points, n: int, gumbel, tau: float = 1.0, comp_key=None):
    """reassign (Alg. 1): returns (picked points, picked components), host
    int arrays in rank order; the prior means of the components are now the
    points'.  gumbel: N standard Gumbel variates; comp_key: K tie keys or None."""
    ptr, N, keep = _points_ptr(points)
    g = _host_f64(gumbel).ravel()
    if g.size != N:
        raise ValueError(f"gumbel needs {N} values, got {g.size}")
    v = None if comp_key is None else _host_f64(comp_key).ravel()
    pts = np.zeros(max(n, 1), dtype=np.int64)
    comps = np.zeros(max(n, 1), dtype=np.int32)
    _check(lib().vbgs_reassign(ctx, ptr, N, int(n), float(tau), _dp(g), None if v is None else _dp(v),
                               pts.ctypes.data_as(C.POINTER(C.c_int64)), comps.ctypes.data_as(C.POINTER(C.c_int))),
           ctx)
    del keep
    return pts[:n], comps[:n]


def vbgs_get_posterior(ctx, K: int) -> dict:
    out = {"alpha": np.zeros(K), "beta": np.zeros(K), "m": np.zeros((K, D)),
           "Winv": np.zeros((K, D, D)), "nu": np.zeros(K)}
    _check(lib().vbgs_get_posterior(ctx, _dp(out["alpha"]), _dp(out["beta"]), _dp(out["m"]),
                                    _dp(out["Winv"]), _dp(out["nu"])), ctx)
    return out


def vbgs_get_stats(ctx, K: int) -> np.ndarray:
    S = np.zeros((K, F))
    _check(lib().vbgs_get_stats(ctx, _dp(S)), ctx)
    return S


def vbgs_set_stats(ctx, S) -> None:
    Sa = _host_f64(S)
    _check(lib().vbgs_set_stats(ctx, _dp(Sa)), ctx)


def vbgs_get_frame_stats(ctx, K: int) -> np.ndarray:
    S = np.zeros((K, F))
    _check(lib().vbgs_get_frame_stats(ctx, _dp(S)), ctx)
    return S


def vbgs_get_lse(ctx, N: int) -> np.ndarray:
    lse = np.zeros(max(N, 1))
    _check(lib().vbgs_get_lse(ctx, _dp(lse), N), ctx)
    return lse[:N]


def vbgs_last_launch_count(ctx) -> int:
    return int(lib().vbgs_last_launch_count(ctx))


def prof_only(*classes: int) -> int:
    """vbgs_profile_enable's mask that times only the given classes."""
    m = 0
    for c in classes:
        m |= 1 << (int(c) + 1)
    return m


def vbgs_profile_enable(ctx, on: bool | int = True) -> None:
    _check(lib().vbgs_profile_enable(ctx, int(on)), ctx)


def vbgs_profile_read(ctx, reset: bool = False) -> dict:
    ms = np.zeros(PROF_COUNT)
    n = np.zeros(PROF_COUNT, dtype=np.int64)
    _check(lib().vbgs_profile_read(ctx, _dp(ms), n.ctypes.data_as(C.POINTER(C.c_int64)), int(reset)), ctx)
    return {lib().vbgs_profile_name(i).decode(): (float(ms[i]), int(n[i])) for i in range(PROF_COUNT)}


def vbgs_profile_pairs(ctx) -> tuple[int, int]:
    a, b = C.c_int64(0), C.c_int64(0)
    _check(lib().vbgs_profile_pairs(ctx, C.byref(a), C.byref(b)), ctx)
    return int(a.value), int(b.value)


def vbgs_profile_replay(ctx, reps: int = 100) -> tuple[float, int, int]:
    """(ms per launch, pairs per launch, pairs exponentiated per launch) of
    the last tensor-core pass-1 launch replayed reps times back to back."""
    ms = np.zeros(1)
    pairs = C.c_int64(0)
    epairs = C.c_int64(0)
    _check(lib().vbgs_profile_replay(ctx, int(reps), _dp(ms), C.byref(pairs), C.byref(epairs)), ctx)
    return float(ms[0]), int(pairs.value), int(epairs.value)


def vbgs_probe_peaks(device: int = 0) -> dict:
    out = np.zeros(4)
    _check(lib().vbgs_probe_peaks(device, _dp(out)), None)
    return {"fp64_tflops": float(out[0]), "fp32_tflops": float(out[1]), "mufu_ex2_gops": float(out[2]),
            "sms": int(out[3])}


def _device_f64(t, shape, what: str):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{what} must be a contiguous float64 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


def vbgs_estep_noalloc(ctx, points, lse_out, dS_out, K: int | None = None) -> None:
    """E-step into caller-owned device buffers with no allocation by the
    library (contiguous float64 CUDA tensors: points N x 6, lse_out N,
    dS_out K x 28).  Results are enqueued on the context's stream.  The
    library itself rejects host pointers; these checks also catch wrong
    shapes and dtypes, which the C ABI cannot see."""
    import torch
    if not isinstance(points, torch.Tensor) or points.dim() != 2:
        raise ValueError("points must be an N x 6 float64 CUDA tensor")
    N = points.shape[0]
    _device_f64(points, (N, D), "points")
    _device_f64(lse_out, (N,), "lse_out")
    if K is not None:
        _device_f64(dS_out, (K, F), "dS_out")
    elif dS_out.dim() != 2 or dS_out.shape[1] != F:
        raise ValueError("dS_out must be K x 28")
    else:
        _device_f64(dS_out, tuple(dS_out.shape), "dS_out")
    _check(lib().vbgs_estep_noalloc(ctx, C.c_void_p(points.data_ptr() if N else None), N,
                                    C.c_void_p(lse_out.data_ptr() if N else None),
                                    C.c_void_p(dS_out.data_ptr())), ctx)


def vbgs_estep_noalloc_raw(ctx, points_ptr: int, N: int, lse_ptr: int, dS_ptr: int) -> int:
    """The C entry point with raw addresses and no checks in Python (returns
    the status code): for tests of the library's own argument checks."""
    return int(lib().vbgs_estep_noalloc(ctx, C.c_void_p(points_ptr or None), int(N), C.c_void_p(lse_ptr or None),
                                        C.c_void_p(dS_ptr or None)))


def vbgs_update_batched(ctxs, points_list, n_iters: int) -> np.ndarray:
    """All scenes' frame updates in one graph launch; returns n_scenes x n_iters ELBO traces."""
    n = len(ctxs)
    keep, ptrs, Ns = [], [], []
    for pts in points_list:
        ptr, N, k = _points_ptr(pts)
        keep.append(k)
        ptrs.append(ptr.value)
        Ns.append(N)
    arr_ctx = (C.c_void_p * n)(*[c.value for c in ctxs])
    arr_pts = (C.c_void_p * n)(*ptrs)
    arr_N = (C.c_int64 * n)(*Ns)
    traces = np.zeros((n, n_iters))
    _check(lib().vbgs_update_batched(arr_ctx, n, arr_pts, arr_N, n_iters, _dp(traces)), None)
    del keep
    return traces


def vbgs_autotune(ctx, points, cache_path: str | None = None) -> tuple[int, int]:
    ptr, N, keep = _points_ptr(points)
    _check(lib().vbgs_autotune(ctx, ptr, N, cache_path.encode() if cache_path else None), ctx)
    del keep
    return vbgs_get_tuning(ctx)


def vbgs_set_tuning(ctx, pass1_tiles: int, pass2_chunks: int) -> None:
    _check(lib().vbgs_set_tuning(ctx, int(pass1_tiles), int(pass2_chunks)), ctx)


def vbgs_get_tuning(ctx) -> tuple[int, int]:
    a, b = C.c_int(0), C.c_int(0)
    _check(lib().vbgs_get_tuning(ctx, C.byref(a), C.byref(b)), ctx)
    return int(a.value), int(b.value)


def _fp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_float))


def vbgs_proposal_report(ctx) -> dict:
    out = np.zeros(11)
    _check(lib().vbgs_proposal_report(ctx, _dp(out)), ctx)
    return dict(zip(PROP_REPORT, out.tolist()))


def vbgs_proposal_config(ctx, epochs: int = 8, learning_rate: float = 3e-3) -> None:
    """Training schedule of the proposal network (epochs 0: not trained)."""
    _check(lib().vbgs_proposal_config(ctx, int(epochs), float(learning_rate)), ctx)


def vbgs_proposal_weights(ctx, set_to=None) -> np.ndarray:
    get = np.zeros(PROP_NPARAM, dtype=np.float32)
    st = None if set_to is None else np.ascontiguousarray(set_to, dtype=np.float32)
    _check(lib().vbgs_proposal_weights(ctx, _fp(get), _fp(st)), ctx)
    return get


def vbgs_proposal_grad(ctx, inputs, labels=None):
    """(loss, grad, top) of the network on B inputs (B x 6 in [-1, 1]) and labels (B x 1024)."""
    x = np.ascontiguousarray(inputs, dtype=np.float32)
    B = x.shape[0]
    q = None if labels is None else np.ascontiguousarray(labels, dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    grad = np.zeros(PROP_NPARAM, dtype=np.float32)
    top = np.zeros((B, 4), dtype=np.int32)
    _check(lib().vbgs_proposal_grad(ctx, _fp(x), _fp(q), B, _fp(loss), _fp(grad),
                                    top.ctypes.data_as(C.POINTER(C.c_int))), ctx)
    return float(loss[0]), grad, top


def vbgs_proposal_clusters(ctx, K: int):
    cent = np.zeros((PROP_CLUSTERS, 6), dtype=np.float32)
    cl = np.zeros(K, dtype=np.int32)
    _check(lib().vbgs_proposal_clusters(ctx, _fp(cent), cl.ctypes.data_as(C.POINTER(C.c_int))), ctx)
    return cent, cl


def vbgs_proposal_bounds(ctx, points, K: int):
    """Certificate bounds (log2 units, N x 1024) of the current posterior at
    host points (N x 6) and each component's cluster (K)."""
    x = np.ascontiguousarray(np.asarray(points, dtype=np.float64)[:, :6])
    ub = np.zeros((x.shape[0], PROP_CLUSTERS), dtype=np.float32)
    cl = np.zeros(K, dtype=np.int32)
    _check(lib().vbgs_proposal_bounds(ctx, _dp(x), x.shape[0], _fp(ub), cl.ctypes.data_as(C.POINTER(C.c_int))), ctx)
    return ub, cl


def vbgs_kmeans(points, centroids, lloyd_iters: int):
    """Lloyd's algorithm from the given centroids (1024 x 6) on K x 6 points:
    returns (centroids, nearest-centroid assignment of the points)."""
    x = np.ascontiguousarray(points, dtype=np.float32)
    if x.ndim != 2 or x.shape[1] != 6:
        raise ValueError("points must be K x 6")
    c = np.array(centroids, dtype=np.float32, copy=True, order="C")
    if c.shape != (PROP_CLUSTERS, 6):
        raise ValueError(f"centroids must be {PROP_CLUSTERS} x 6")
    cl = np.zeros(max(x.shape[0], 1), dtype=np.int32)
    _check(lib().vbgs_kmeans(_fp(x) if x.size else None, x.shape[0], _fp(c), int(lloyd_iters),
                             cl.ctypes.data_as(C.POINTER(C.c_int))), None)
    return c, cl[:x.shape[0]]


def camera_array(cam: dict) -> np.ndarray:
    """The 13 doubles of vbgs_render's camera from a view dict (o, Rwc, f)."""
    return np.concatenate([np.asarray(cam["o"], dtype=np.float64).ravel(),
                           np.asarray(cam["Rwc"], dtype=np.float64).ravel(), [float(cam["f"])]])


def vbgs_render(ctx, cam: dict, reference=None, want_image: bool = True):
    """Render the posterior at a camera (dict with o, Rwc, f, width, height);
    returns (image H x W x 3 float32 or None, PSNR against reference or None,
    device ms)."""
    W, H = int(cam["width"]), int(cam["height"])
    c = camera_array(cam)
    img = np.zeros((H, W, 3), dtype=np.float32) if want_image else None
    ref = None
    if reference is not None:
        ref = np.ascontiguousarray(reference, dtype=np.float32)
        if ref.shape != (H, W, 3):
            raise ValueError(f"reference must be {H} x {W} x 3")
    p = np.zeros(1)
    ms = np.zeros(1)
    _check(lib().vbgs_render(ctx, _dp(c), W, H, _fp(img), _fp(ref), _dp(p) if ref is not None else None, _dp(ms)),
           ctx)
    return img, (float(p[0]) if ref is not None else None), float(ms[0])


def vbgs_set_precision_knobs(ctx, knobs: int) -> None:
    """Leave out the lo terms of the set bits (KNOBS) in the tensor-core passes."""
    _check(lib().vbgs_set_precision_knobs(ctx, int(knobs)), ctx)


def vbgs_get_precision_knobs(ctx) -> int:
    return int(lib().vbgs_get_precision_knobs(ctx))


def vbgs_set_wait_limit(cycles: int) -> None:
    """Limit (SM cycles) of the waits between warp roles of the tensor-core
    kernels on the current device; <= 0 restores the default."""
    _check(lib().vbgs_set_wait_limit(int(cycles)), None)


def vbgs_last_error(ctx=None) -> str:
    return lib().vbgs_last_error(ctx).decode(errors="replace")


def vbgs_destroy(ctx) -> None:
    if ctx:
        lib().vbgs_destroy(ctx)


class Model:
    """One VBGS mixture on the GPU (owns a vbgs_ctx)."""

    def __init__(self, prior: dict | None, precision: str | int = "fp64", cuda_stream: int | None = None,
                 flags: int = 0, checks: bool = False, autotune_cache: str | None = None, seed: int = 0,
                 _ctx=None, _K: int = 0):
        self.ctx = None
        if _ctx is not None:        # Model.load
            self.K, self.ctx = int(_K), _ctx
            return
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.K = int(np.asarray(prior["m0"]).shape[0])
        self.ctx = vbgs_init(prior["alpha0"], prior["beta0"], prior["nu0"], prior["m0"], prior["W0"],
                             p, cuda_stream, flags, checks, autotune_cache, seed)

    @classmethod
    def load(cls, path: str, cuda_stream: int | None = None, checks: bool = False,
             autotune_cache: str | None = None) -> "Model":
        """A model resumed from a file vbgs_save_state wrote."""
        ctx = vbgs_load_state(path, cuda_stream, checks, autotune_cache)
        with open(path, "rb") as f:
            K = int(np.frombuffer(f.read(16), dtype=np.int32)[3])   # magic (8 bytes), version, K
        return cls(None, _ctx=ctx, _K=K)

    def save(self, path: str) -> None:
        vbgs_save_state(self.ctx, path)

    def render(self, cam: dict, reference=None, want_image: bool = True):
        return vbgs_render(self.ctx, cam, reference, want_image)

    def update(self, points, n_iters: int) -> np.ndarray:
        return vbgs_update(self.ctx, points, n_iters)

    def elbo(self, points, want_lse: bool = False):
        return vbgs_elbo(self.ctx, points, want_lse)

    def reassign(self, points, n: int, gumbel, tau: float = 1.0, comp_key=None):
        if comp_key is not None and np.asarray(comp_key).size != self.K:
            raise ValueError(f"comp_key needs {self.K} values")
        return vbgs_reassign(self.ctx, points, n, gumbel, tau, comp_key)

    def posterior(self) -> dict:
        return vbgs_get_posterior(self.ctx, self.K)

    def stats(self) -> np.ndarray:
        return vbgs_get_stats(self.ctx, self.K)

    def set_stats(self, S) -> None:
        vbgs_set_stats(self.ctx, S)

    def frame_stats(self) -> np.ndarray:
        return vbgs_get_frame_stats(self.ctx, self.K)

    def lse(self, N: int) -> np.ndarray:
        return vbgs_get_lse(self.ctx, N)

    def launches(self) -> int:
        return vbgs_last_launch_count(self.ctx)

    def profile(self, on: bool | int = True) -> None:
        vbgs_profile_enable(self.ctx, on)

    def profile_read(self, reset: bool = False) -> dict:
        return vbgs_profile_read(self.ctx, reset)

    def profile_pairs(self) -> tuple[int, int]:
        return vbgs_profile_pairs(self.ctx)

    def close(self) -> None:
        if self.ctx:
            vbgs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
