"""GPU parity at the learned-proposal workload's size: K = 200,000
components, room frames of 96 x 96 points, from the FP64 oracle's own state
after two frames (2 CAVI iterations each), one iteration on the next frame
in every form and with the learned proposal, against `oracle.cavi_frame`.

Bounds: FP64 1e-10; the reduced and proposal forms the stated targets, 1e-3
per statistic array and 1e-4 on the ELBO (Eq. relerr).  Per component
(components with Delta N_k >= 1): FP32 1e-3 and FP16x3 1e-2 -- at this K the
components are tighter than at K = 50,000 (precisions up to ~4x higher in a
tile of the same point spread), so the largest expanded logit term and with
it the logit error of the hi/lo form grow by that factor (the K = 50,000
bound is 2e-3); the proposal form's scoring is FP32, and its certificate
lets each point miss up to 1e-3 of its mass, so its bound is 1e-3 plus the
FP32 bound's share, 2e-3 per point of mass, checked as a total
sum_k |dN_k| <= 2e-3 N.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_08499_gb300 import synth

pytestmark = pytest.mark.gpu

K = 200_000
SEED = 5
TOL = {"fp64": dict(stat=1e-10, elbo=1e-10, comp=1e-10), "fp32": dict(stat=1e-3, elbo=1e-4, comp=1e-3),
       "fp16x3": dict(stat=1e-3, elbo=1e-4, comp=1e-2)}


@pytest.fixture(scope="module")
def V():
    from paper_2603_08499_gb300 import build
    build.build()
    from paper_2603_08499_gb300 import vbgs
    return vbgs


@pytest.fixture(scope="module")
def state():
    room = synth.Room(SEED)
    pr = synth.room_prior(K, seed=SEED)
    S = np.zeros((K, 28))
    for t in range(2):
        X = synth.room_frame(t, seed=SEED, width=96, height=96, room=room)
        S = O.cavi_frame(X, pr, S, 2)[1]
    X2 = synth.room_frame(2, seed=SEED, width=96, height=96, room=room)
    e_ref, _, lse_ref, dS_ref = O.cavi_frame(X2, pr, S, 1)
    return dict(prior=pr, S=S, X=X2, elbo=e_ref, lse=lse_ref, dS=dS_ref)


def _errors(trace, dS, st):
    ref = st["dS"]
    sel = ref[:, 0] >= 1.0
    errs = {"elbo": O.relerr(trace, st["elbo"]), "N": O.relerr(dS[:, 0], ref[:, 0]),
            "S1": O.relerr(dS[:, 1:7], ref[:, 1:7]), "S2": O.relerr(dS[:, 7:], ref[:, 7:]),
            "comp": float(np.max(np.abs(dS[sel, 0] - ref[sel, 0]) / ref[sel, 0]))}
    return errs


@pytest.mark.parametrize("form", ["fp64", "fp32", "fp16x3"])
def test_k200000_one_iteration_against_oracle(V, state, form):
    import torch
    m = V.Model(state["prior"], form)
    m.set_stats(state["S"])
    tr = m.update(torch.from_numpy(state["X"]).cuda(), 1)
    errs = _errors(tr, m.frame_stats(), state)
    m.close()
    print(f"\nK=200000 {form}: {errs}")
    tol = TOL[form]
    assert errs["elbo"] <= tol["elbo"], errs
    for k in ("N", "S1", "S2"):
        assert errs[k] <= tol["stat"], (k, errs)
    assert errs["comp"] <= tol["comp"], errs


@pytest.mark.parametrize("form", ["fp32", "fp16x3"])
def test_k200000_proposal_against_oracle(V, state, form):
    import torch
    X = state["X"]
    m = V.Model(state["prior"], form, flags=V.VBGS_FLAG_PROPOSAL)
    m.set_stats(state["S"])
    tr = m.update(torch.from_numpy(X).cuda(), 1)
    dS = m.frame_stats()
    rep = V.vbgs_proposal_report(m.ctx)
    m.close()
    errs = _errors(tr, dS, state)
    print(f"\nK=200000 proposal ({form} fallback): {errs} report {rep}")
    assert rep["audit_max_missed"] <= 1e-3
    assert errs["elbo"] <= 1e-4, errs
    for k in ("N", "S1", "S2"):
        assert errs[k] <= 1e-3, (k, errs)
    assert np.abs(dS[:, 0] - state["dS"][:, 0]).sum() <= 2e-3 * X.shape[0]
