"""GPU tests of vbgs_estep_noalloc, the E-step for callers that cannot
allocate device memory (their device memory belongs to a host runtime's own
pool or a fixed budget, or they cannot take an allocation mid-frame).  The
entry point takes its scratch from the library's static device array, so
consecutive calls share it: both calls below must match the regular context
path, the second with fewer points than the first.  This file is collected
last so that a failure here stops a -x run only after every other test."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_08499_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    from paper_2603_08499_gb300 import build
    build.build()
    from paper_2603_08499_gb300 import vbgs
    return vbgs


# FP64 contexts run the FP64 E-step: FP64 rounding only.  FP32, FP16X3 and
# BF16X3 contexts run the FP32 CUDA-core E-step: the FP32 form's tolerances
# (FP32 logits, ~1e-7 relative, over one iteration) against the FP64 result.
TOL = {"fp64": (1e-10, 1e-10), "fp32": (1e-4, 1e-3), "fp16x3": (1e-4, 1e-3), "bf16x3": (1e-4, 1e-3)}


@pytest.mark.parametrize("form", ["fp64", "fp32", "fp16x3", "bf16x3"])
def test_noalloc_estep_matches_context_path_on_two_calls(V, form):
    import torch
    room = synth.Room(seed=5)
    K = 3000
    pr = synth.room_prior(K, seed=5)
    base = V.Model(pr, "fp64")
    base.update(synth.room_frame(0, seed=5, width=80, height=80, room=room), 2)
    S = base.stats()
    base.close()
    na = V.Model(pr, form)
    na.set_stats(S)
    frames = [synth.room_frame(1, seed=5, width=120, height=120, room=room),
              synth.room_frame(2, seed=5, width=64, height=64, room=room)]
    tol_lse, tol_stat = TOL[form]
    for X in frames:
        # the regular context path's first E-step of the same state (FP64)
        ref = V.Model(pr, "fp64")
        ref.set_stats(S)
        ref.update(X, 1)
        lse_ref = ref.lse(X.shape[0])
        dS_ref = ref.frame_stats()
        ref.close()
        lse = torch.full((X.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
        dS = torch.full((K, 28), float("nan"), dtype=torch.float64, device="cuda")
        V.vbgs_estep_noalloc(na.ctx, torch.from_numpy(X).cuda(), lse, dS, K)
        torch.cuda.synchronize()
        assert O.relerr(lse.cpu().numpy(), lse_ref) <= tol_lse
        got = dS.cpu().numpy()
        for sl in (slice(0, 1), slice(1, 7), slice(7, 28)):
            assert O.relerr(got[:, sl], dS_ref[:, sl]) <= tol_stat
    assert np.array_equal(na.stats(), S)
    na.close()


def test_noalloc_rejects_host_memory(V):
    """Host arrays are refused on the host, before any launch."""
    import torch
    X, pr = synth.c1_workload(seed=4, N=64, K=20)
    m = V.Model(pr, "fp64")
    Xh = np.ascontiguousarray(X)
    lse_h = np.zeros(64)
    dS_h = np.zeros((20, 28))
    Xd = torch.from_numpy(X).cuda()
    lse_d = torch.zeros(64, dtype=torch.float64, device="cuda")
    dS_d = torch.zeros((20, 28), dtype=torch.float64, device="cuda")
    for pts, l, d in ((Xh.ctypes.data, lse_d.data_ptr(), dS_d.data_ptr()),
                      (Xd.data_ptr(), lse_h.ctypes.data, dS_d.data_ptr()),
                      (Xd.data_ptr(), lse_d.data_ptr(), dS_h.ctypes.data)):
        assert V.vbgs_estep_noalloc_raw(m.ctx, pts, 64, l, d) == V.VBGS_EINVAL
        assert "device memory" in V.vbgs_last_error(m.ctx)
    with pytest.raises(ValueError):
        V.vbgs_estep_noalloc(m.ctx, Xd, lse_d[:10], dS_d, 20)
    with pytest.raises(ValueError):
        V.vbgs_estep_noalloc(m.ctx, Xd, lse_d, dS_d.float(), 20)
    assert np.all(dS_h == 0) and np.all(lse_h == 0)
    m.close()


def test_noalloc_rejects_sizes_beyond_the_scratch_array(V):
    import torch
    _, pr = synth.c1_workload(seed=3, N=10, K=50)
    m = V.Model(pr, "fp64")
    N = 2_000_000   # 8 N doubles alone exceed the 24 MiB array
    X = torch.zeros((N, 6), dtype=torch.float64, device="cuda")
    lse = torch.empty(N, dtype=torch.float64, device="cuda")
    dS = torch.empty((50, 28), dtype=torch.float64, device="cuda")
    with pytest.raises(V.VbgsError) as e:
        V.vbgs_estep_noalloc(m.ctx, X, lse, dS, 50)
    assert e.value.code == V.VBGS_EINVAL and "scratch array" in str(e.value)
    m.close()
