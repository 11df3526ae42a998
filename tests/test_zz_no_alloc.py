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


def test_noalloc_estep_matches_context_path_on_two_calls(V):
    import torch
    room = synth.Room(seed=5)
    K = 3000
    pr = synth.room_prior(K, seed=5)
    base = V.Model(pr, "fp64")
    base.update(synth.room_frame(0, seed=5, width=80, height=80, room=room), 2)
    S = base.stats()
    base.close()
    na = V.Model(pr, "fp64")
    na.set_stats(S)
    frames = [synth.room_frame(1, seed=5, width=120, height=120, room=room),
              synth.room_frame(2, seed=5, width=64, height=64, room=room)]
    for X in frames:
        ref = V.Model(pr, "fp64")
        ref.set_stats(S)
        ref.update(X, 1)
        lse_ref = ref.lse(X.shape[0])
        dS_ref = ref.frame_stats()
        ref.close()
        lse = torch.full((X.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
        dS = torch.full((K, 28), float("nan"), dtype=torch.float64, device="cuda")
        V.vbgs_estep_noalloc(na.ctx, torch.from_numpy(X).cuda(), lse, dS)
        torch.cuda.synchronize()
        assert O.relerr(lse.cpu().numpy(), lse_ref) <= 1e-10
        got = dS.cpu().numpy()
        for sl in (slice(0, 1), slice(1, 7), slice(7, 28)):
            assert O.relerr(got[:, sl], dS_ref[:, sl]) <= 1e-10
    assert np.array_equal(na.stats(), S)
    na.close()


def test_noalloc_rejects_sizes_beyond_the_scratch_array(V):
    import torch
    _, pr = synth.c1_workload(seed=3, N=10, K=50)
    m = V.Model(pr, "fp64")
    N = 2_000_000   # 8 N doubles alone exceed the 24 MiB array
    X = torch.zeros((N, 6), dtype=torch.float64, device="cuda")
    lse = torch.empty(N, dtype=torch.float64, device="cuda")
    dS = torch.empty((50, 28), dtype=torch.float64, device="cuda")
    with pytest.raises(V.VbgsError) as e:
        V.vbgs_estep_noalloc(m.ctx, X, lse, dS)
    assert e.value.code == V.VBGS_EINVAL and "scratch array" in str(e.value)
    m.close()
