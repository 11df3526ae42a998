"""GPU parity of vbgs_reassign (Alg. 1, the step before fit) through the C
ABI against the oracle's reassign on the same seeded inputs.

Index work is compared bit for bit: the picked components (their order
depends only on S_past and the tie keys, FP64 on both sides) and, for the
FP64 form, the picked points (keys from an lse within 1e-10 of the oracle's;
if the n-th and (n+1)-th oracle keys lie closer than that margin, validity is
checked instead).  The FP16 hi/lo form's point picks are checked for
validity: every point whose oracle key clears the boundary band (twice the
measured lse error) is picked as the oracle picks it, and the picks are
exactly the top n of the keys the kernel computes from its own lse.  The new
prior means, and a CAVI frame from them, match the oracle."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from oracle import reassign as RA
from paper_2603_08499_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    from paper_2603_08499_gb300 import build
    build.build()
    from paper_2603_08499_gb300 import vbgs
    return vbgs


def _state(X, pr, frac=0.5, iters=3):
    """S_past from the oracle after one frame on a part of the points, so
    that some components are visited and many are not."""
    K = pr["m0"].shape[0]
    _, S, _, _ = O.cavi_frame(X[: int(X.shape[0] * frac)], pr, np.zeros((K, 28)), iters)
    return S


def _top_n_from(lse, g, tau, n):
    """Top n of g - lse / tau, ties to the lower index (a plain restatement
    for the validity check, not the oracle)."""
    keys = g - lse * (1.0 / tau)
    return np.lexsort((np.arange(keys.size), -keys))[:n]


def _check_point_picks(pts, lse_gpu, lse_ref, g, tau, n, exact_margin=None):
    keys_ref = RA.point_keys(lse_ref, g, tau)
    s = np.sort(keys_ref)[::-1]
    # the kernel's picks are the top n of the keys from its own lse
    assert np.array_equal(pts, _top_n_from(lse_gpu, g, tau, n))
    if exact_margin is not None and (n == keys_ref.size or s[n - 1] - s[n] > exact_margin):
        assert np.array_equal(pts, RA.pick_points(keys_ref, n))
        return
    band = 2.0 * np.max(np.abs(lse_gpu - lse_ref)) / tau + 1e-12
    thr = s[n - 1]
    sure_in = np.flatnonzero(keys_ref > thr + band)
    assert set(sure_in.tolist()) <= set(pts.tolist())
    assert np.all(keys_ref[pts] >= thr - band)


@pytest.mark.parametrize("n,use_key", [(1, False), (40, True), (197, True)])
def test_reassign_fp64_matches_oracle(V, n, use_key):
    X, pr = synth.c1_workload(seed=31, N=2_345, K=197)
    S = _state(X, pr)
    rng = np.random.default_rng(3)
    g = rng.gumbel(size=X.shape[0])
    v = rng.random(197) if use_key else None
    m = V.Model(pr, "fp64")
    m.set_stats(S)
    pts, comps = m.reassign(X, n, g, tau=1.0, comp_key=v)
    ref_pts, ref_comps, m0_ref, lse_ref = RA.reassign(X, pr, S, n, g, 1.0, v)
    assert np.array_equal(comps, ref_comps)
    lse_gpu = m.lse(X.shape[0])
    assert O.relerr(lse_gpu, lse_ref) <= 1e-10
    keys = RA.point_keys(lse_ref, g, 1.0)
    _check_point_picks(pts, lse_gpu, lse_ref, g, 1.0, n, exact_margin=1e-9 * max(1.0, np.abs(keys).max()))
    # the posterior now has the new prior means; S_past is unchanged
    pr_new = dict(pr, m0=np.array(pr["m0"], dtype=np.float64))
    pr_new["m0"][comps] = X[pts]
    post, post_ref = m.posterior(), O.mstep(pr_new, S)
    assert O.relerr(post["m"], post_ref["m"]) <= 1e-12
    assert np.array_equal(m.stats(), S)
    # a CAVI frame from the new prior (the carried prior must not be reused)
    trace = m.update(X, 3)
    e_ref, S_ref, _, _ = O.cavi_frame(X, pr_new, S, 3)
    for i in range(3):
        assert O.relerr(trace[i], e_ref[i]) <= 1e-10
    assert O.relerr(m.stats(), S_ref) <= 1e-10
    m.close()


def test_reassign_after_frames_does_not_reuse_the_carried_prior(V):
    """Two frames (the second would start from the carried posterior), then
    reassign, then a third frame: equal to the oracle stream with the new
    prior from the third frame on.  S_past here is the GPU's own: components
    far from every point have N_k exactly 0 on the GPU (their pairs are
    certified negligible and skipped) and about 1e-40 in the oracle, so the
    order among them is not unique; the picks are checked for validity (the
    least-used up to that slack, points by the boundary band) and the third
    frame is compared for the choice made."""
    X, pr = synth.c1_workload(seed=33, N=3_000, K=300)
    frames = [X[:1000], X[1000:2000], X[2000:]]
    m = V.Model(pr, "fp64")
    S = np.zeros((300, 28))
    for F in frames[:2]:
        m.update(F, 2)
        _, S, _, _ = O.cavi_frame(F, pr, S, 2)
    assert O.relerr(m.stats(), S) <= 1e-10
    rng = np.random.default_rng(4)
    g = rng.gumbel(size=1000)
    pts, comps = m.reassign(frames[2], 25, g, tau=0.5)
    _, _, _, lse_ref = RA.reassign(frames[2], pr, S, 25, g, 0.5)
    counts = S[:, 0]
    nth = np.sort(counts)[24]
    assert len(set(comps.tolist())) == 25
    assert np.all(counts[comps] <= nth + 1e-9 * max(1.0, counts.max()))
    _check_point_picks(pts, m.lse(1000), lse_ref, g, 0.5, 25)
    pr_new = dict(pr, m0=np.array(pr["m0"], dtype=np.float64))
    pr_new["m0"][comps] = frames[2][pts]
    trace = m.update(frames[2], 2)
    e_ref, S_ref, _, _ = O.cavi_frame(frames[2], pr_new, S, 2)
    assert O.relerr(trace[-1], e_ref[-1]) <= 1e-10
    assert O.relerr(m.stats(), S_ref) <= 1e-10
    m.close()


def test_reassign_fp16x3_picks_are_valid(V):
    X, pr = synth.c1_workload(seed=32, N=5_000, K=1_500)
    S = _state(X, pr, frac=0.4)
    rng = np.random.default_rng(5)
    g = rng.gumbel(size=X.shape[0])
    v = rng.random(1_500)
    m = V.Model(pr, "fp16x3")
    m.set_stats(S)
    pts, comps = m.reassign(X, 120, g, tau=2.0, comp_key=v)
    _, ref_comps, _, lse_ref = RA.reassign(X, pr, S, 120, g, 2.0, v)
    assert np.array_equal(comps, ref_comps)
    lse_gpu = m.lse(X.shape[0])
    assert O.relerr(lse_gpu, lse_ref) <= 1e-3
    _check_point_picks(pts, lse_gpu, lse_ref, g, 2.0, 120)
    m.close()


def test_reassign_full_size_room_frame(V):
    """The benchmark's shape: K = 50,000 components, a room frame of up to
    40,000 points, n = 500.  Components against the oracle's order of the same
    S_past (a valid synthetic state with most components unvisited); points
    against the top 500 of the kernel's own keys, and the lse of 32 sampled
    picked points against the oracle one by one."""
    import torch
    K, n = 50_000, 500
    room = synth.Room(seed=7)
    pr = synth.room_prior(K, seed=7)
    X = synth.room_frame(0, seed=7, room=room)
    rng = np.random.default_rng(6)
    S = np.zeros((K, 28))
    vis = rng.choice(K, size=6_000, replace=False)
    Nk = rng.uniform(0.5, 50.0, size=vis.size)
    mu = np.asarray(pr["m0"])[vis] + 0.01 * rng.standard_normal((vis.size, 6))
    S[vis, 0] = Nk
    S[vis, 1:7] = Nk[:, None] * mu
    iu = np.triu_indices(6)
    cov = np.einsum("ni,nj->nij", mu, mu) + 1e-4 * np.eye(6)
    S[vis, 7:] = Nk[:, None] * cov[:, iu[0], iu[1]]
    g = rng.gumbel(size=X.shape[0])
    v = rng.random(K)
    m = V.Model(pr, "fp16x3")
    m.set_stats(S)
    Xd = torch.from_numpy(X).cuda()
    pts, comps = m.reassign(Xd, n, g, tau=1.0, comp_key=v)
    assert np.array_equal(comps, RA.pick_components(S[:, 0], n, v))
    assert set(comps.tolist()).isdisjoint(vis.tolist())
    lse_gpu = m.lse(X.shape[0])
    assert np.array_equal(pts, _top_n_from(lse_gpu, g, 1.0, n))
    sample = pts[rng.choice(n, size=32, replace=False)]
    lse_ref, _, _ = O.estep_stats(X[sample], O.mstep(pr, S))
    assert np.max(np.abs(lse_gpu[sample] - lse_ref) / np.maximum(1.0, np.abs(lse_ref))) <= 1e-3
    post = m.posterior()
    assert np.allclose(post["m"][comps], X[pts], rtol=0, atol=1e-12)
    m.close()


def test_reassign_edges_and_errors_leave_the_prior_unchanged(V):
    X, pr = synth.c1_workload(seed=34, N=300, K=50)
    m = V.Model(pr, "fp64")
    before = m.posterior()["m"].copy()
    g = np.random.default_rng(7).gumbel(size=300)
    pts, comps = m.reassign(X, 0, g)
    assert pts.size == 0 and comps.size == 0
    for bad in (dict(n=51), dict(n=-1), dict(n=5, tau=0.0), dict(n=5, tau=-1.0)):
        with pytest.raises(V.VbgsError) as e:
            m.reassign(X, bad["n"], g, tau=bad.get("tau", 1.0))
        assert e.value.code == V.VBGS_EINVAL
    gbad = g.copy()
    gbad[17] = np.inf
    with pytest.raises(V.VbgsError):
        m.reassign(X, 5, gbad)
    Xbad = X.copy()
    Xbad[3, 2] = np.nan
    with pytest.raises(V.VbgsError):
        m.reassign(Xbad, 5, g)
    assert np.array_equal(m.posterior()["m"], before)
    # n = N = K on a tiny case: every point and every component
    Xs, prs = synth.c1_workload(seed=35, N=7, K=7)
    ms = V.Model(prs, "fp64")
    gs = np.random.default_rng(8).gumbel(size=7)
    pts, comps = ms.reassign(Xs, 7, gs)
    ref_pts, ref_comps, _, _ = RA.reassign(Xs, prs, np.zeros((7, 28)), 7, gs)
    assert np.array_equal(comps, ref_comps) and sorted(pts.tolist()) == list(range(7))
    ms.close()
    m.close()


def test_reassign_device_points_equal_host_points(V):
    import torch
    X, pr = synth.c1_workload(seed=36, N=1_000, K=120)
    S = _state(X, pr)
    g = np.random.default_rng(9).gumbel(size=1_000)
    out = []
    for pts_in in (X, torch.from_numpy(X).cuda()):
        m = V.Model(pr, "fp16x3")
        m.set_stats(S)
        out.append(m.reassign(pts_in, 30, g))
        out.append(m.posterior()["m"])
        m.close()
    assert np.array_equal(out[0][0], out[2][0]) and np.array_equal(out[0][1], out[2][1])
    assert np.array_equal(out[1], out[3])
