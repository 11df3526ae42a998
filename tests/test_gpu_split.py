"""GPU parity of the split model (VBGS_FLAG_SPLIT; Sec. 2.1.2, Fig. 3: a
spatial and a colour Normal-Wishart per component, one Dirichlet) through
the C ABI against the split-model oracle on the same seeded inputs:
statistics, ELBO trace and lse within the forms' tolerances (FP64 1e-10;
FP16 hi/lo 1e-3 per statistic array, 1e-4 on the ELBO), the posterior's
block-diagonal W^-1 (cross blocks exactly zero), a second frame from the
carried prior, and the prior's argument check."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from oracle import split as SP
from paper_2603_08499_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-10, 1e-10, 1e-10), "fp16x3": (1e-3, 1e-4, 1e-3)}   # stats, ELBO, lse


@pytest.fixture(scope="module")
def V():
    from paper_2603_08499_gb300 import build
    build.build()
    from paper_2603_08499_gb300 import vbgs
    return vbgs


def _errs(S, S_ref):
    return [O.relerr(S[:, 0], S_ref[:, 0]), O.relerr(S[:, 1:7], S_ref[:, 1:7]), O.relerr(S[:, 7:], S_ref[:, 7:])]


@pytest.mark.parametrize("form", ["fp64", "fp16x3"])
def test_split_model_frames_match_oracle(V, form):
    X, pr = synth.c1_workload(seed=41, N=2_345, K=197)
    tol_s, tol_e, tol_l = TOL[form]
    m = V.Model(pr, form, flags=V.VBGS_FLAG_SPLIT)
    S = np.zeros((197, 28))
    for t, F in enumerate((X[:1_200], X[1_200:])):      # the second frame starts from the carried prior
        trace = m.update(F, 4)
        e_ref, S, lse_ref, _ = SP.cavi_frame(F, pr, S, 4)
        for i in range(4):
            assert O.relerr(trace[i], e_ref[i]) <= tol_e, (t, i, trace[i], e_ref[i])
        assert max(_errs(m.stats(), S)) <= tol_s, (t, _errs(m.stats(), S))
        assert O.relerr(m.lse(F.shape[0]), lse_ref) <= tol_l
    post = m.posterior()
    q_s, q_c = SP.mstep(pr, S)
    assert np.all(post["Winv"][:, :3, 3:] == 0) and np.all(post["Winv"][:, 3:, :3] == 0)
    if form == "fp64":
        assert O.relerr(post["Winv"][:, :3, :3], q_s["Winv"]) <= 1e-10
        assert O.relerr(post["Winv"][:, 3:, 3:], q_c["Winv"]) <= 1e-10
        assert O.relerr(post["m"][:, :3], q_s["m"]) <= 1e-10 and O.relerr(post["m"][:, 3:], q_c["m"]) <= 1e-10
    m.close()


def test_split_model_differs_from_the_joint_model(V):
    X, pr = synth.c1_workload(seed=42, N=800, K=40)
    a = V.Model(pr, "fp64", flags=V.VBGS_FLAG_SPLIT)
    b = V.Model(pr, "fp64")
    ta, tb = a.update(X, 3), b.update(X, 3)
    e_split, _, _, _ = SP.cavi_frame(X, pr, np.zeros((40, 28)), 3)
    e_joint, _, _, _ = O.cavi_frame(X, pr, np.zeros((40, 28)), 3)
    assert O.relerr(ta, e_split) <= 1e-10 and O.relerr(tb, e_joint) <= 1e-10
    assert O.relerr(ta, tb) > 1e-6
    a.close()
    b.close()


def test_split_model_prior_check(V):
    _, pr = synth.c1_workload(seed=43, N=10, K=4)
    pr = dict(pr, nu0=4.0)                   # a valid 3-D Wishart, not a 6-D one
    with pytest.raises(V.VbgsError) as e:
        V.Model(pr, "fp64")
    assert e.value.code == V.VBGS_EINVAL
    m = V.Model(pr, "fp64", flags=V.VBGS_FLAG_SPLIT)
    m.close()
    with pytest.raises(V.VbgsError):
        V.Model(dict(pr, nu0=2.0), "fp64", flags=V.VBGS_FLAG_SPLIT)
