"""GPU tests of the learned-proposal E-step (k-means clusters, MLP, missed-mass
certificate, candidate E-step) through the C ABI, against the FP64 oracles:
the MLP gradient against oracle/mlp.py, the integer decisions (top-4 and the
k-means assignment) by their defining rule, the certificate as an upper bound
of every cluster's exact mass, and a proposal iteration against the exact
CAVI iteration of oracle/ from the same state, with error bounds derived from
the certificate's 1e-3 missed-mass threshold."""
from __future__ import annotations

import numpy as np
import pytest
from scipy.special import digamma, logsumexp

from oracle import mlp as M
from oracle import oracle as O
from paper_2603_08499_gb300 import synth

pytestmark = pytest.mark.gpu

LN2 = np.log(2.0)


@pytest.fixture(scope="module")
def V():
    from paper_2603_08499_gb300 import build
    build.build()
    from paper_2603_08499_gb300 import vbgs
    return vbgs


def bf16(a):
    """Round-to-nearest-even to BF16 (the network's weight format)."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32)


@pytest.fixture(scope="module")
def room_state():
    """Two room frames of CAVI by the FP64 oracle (K = 8,000, 96 x 96 frames)
    and the next frame: the state the proposal tests start from."""
    room = synth.Room(seed=21)
    pr = synth.room_prior(8_000, seed=21)
    S = np.zeros((8_000, 28))
    for t in range(2):
        X = synth.room_frame(t, seed=21, width=96, height=96, room=room)
        S = O.cavi_frame(X, pr, S, 3)[1]
    X2 = synth.room_frame(2, seed=21, width=96, height=96, room=room)
    return pr, S, X2


def test_mlp_gradient_matches_fp64_oracle(V):
    _, pr = synth.c1_workload(seed=31, N=10, K=2_000)
    m = V.Model(pr, "fp32", flags=V.VBGS_FLAG_PROPOSAL)
    rng = np.random.default_rng(31)
    w = V.vbgs_proposal_weights(m.ctx)
    # biases away from zero so every block of the gradient is exercised
    w = w.copy()
    w[128 * 6:128 * 7] = rng.normal(0, 0.1, 128)
    V.vbgs_proposal_weights(m.ctx, w)
    x = rng.uniform(-1, 1, (333, 6)).astype(np.float32)
    q = rng.dirichlet(np.full(1024, 0.05), size=333).astype(np.float32)
    loss, g, top = V.vbgs_proposal_grad(m.ctx, x, q)
    wb = bf16(w).astype(np.float64)
    # FP32 accumulation against FP64: relative error of the whole gradient
    assert abs(loss - M.loss(wb, x, q)) <= 1e-5 * abs(M.loss(wb, x, q))
    assert O.relerr(g, M.grad(wb, x, q)) <= 1e-4
    # top-4: the chosen clusters are the 4 largest logits (up to FP32 ties)
    z = M.forward(wb, x)[2]
    zs = np.sort(z, axis=1)[:, ::-1]
    for i in range(x.shape[0]):
        assert len(set(top[i])) == 4
        assert np.all(z[i, top[i]] >= zs[i, 3] - 1e-4 * (1 + abs(zs[i, 3])))
    m.close()


def test_kmeans_assignment_is_nearest_centroid(V, room_state):
    pr, S, _ = room_state
    K = pr["m0"].shape[0]
    m = V.Model(pr, "fp32", flags=V.VBGS_FLAG_PROPOSAL)
    m.set_stats(S)
    for _ in range(3):
        cent, cl = V.vbgs_proposal_clusters(m.ctx, K)
    # clustering features: posterior mean, colour scaled by a fifth of the
    # largest extent of the padded prior-mean box
    lo, hi = pr["m0"][:, :3].min(0), pr["m0"][:, :3].max(0)
    csc = np.float32(0.2 * np.max(1.2 * (hi - lo) + 2e-6))
    mean = O.mstep(pr, S)["m"].astype(np.float32)
    feat = mean.copy()
    feat[:, 3:] *= csc
    d2 = ((feat[:, None, :].astype(np.float64) - cent[None].astype(np.float64)) ** 2).sum(-1)
    own = d2[np.arange(K), cl]
    assert np.all(own <= d2.min(1) * (1 + 1e-5) + 1e-9)
    assert np.all((cl >= 0) & (cl < 1024))
    m.close()


def _nearest(X, C):
    """Nearest centroid from the definition (FP64 distances of the FP32
    values, ties to the lower index) and the gap to the nearest centroid at
    another position: assignments whose gap is within FP32 rounding of the
    distances may differ between FP32 and FP64 arithmetic."""
    d2 = ((X[:, None, :].astype(np.float64) - C[None].astype(np.float64)) ** 2).sum(-1)
    a = d2.argmin(1)
    best = d2[np.arange(X.shape[0]), a]
    same_pos = np.all(C[None, :, :] == C[a][:, None, :], axis=2)
    other = np.where(same_pos, np.inf, d2).min(1)
    ambiguous = other - best <= 1e-5 * (1.0 + best)
    return a, ambiguous


def _kmeans_case(seed=31, K=20_000):
    """Points in 300 blobs; warm-start centroids drawn from the points, with
    an exact duplicate pair (the tie rule) and two far-away centroids that no
    point is nearest to (empty clusters keep their centroids)."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-3, 3, (300, 6))
    X = (centres[rng.integers(0, 300, K)] + 0.2 * rng.standard_normal((K, 6))).astype(np.float32)
    C0 = X[rng.choice(K, 1024, replace=False)].copy()
    C0[700] = C0[5]
    C0[1000] = 1e3
    C0[1023] = -1e3
    return X, C0


def test_kmeans_lloyd_step_against_definition(V):
    """One Lloyd step against its definition: every point to its nearest
    centroid (ties to the lower index), every centroid to the mean of its
    members, empty clusters keep their centroids; the returned assignment is
    the nearest of the returned centroids."""
    X, C0 = _kmeans_case()
    C1, cl = V.vbgs_kmeans(X, C0, 1)
    a0, amb0 = _nearest(X, C0)
    scale = float(np.abs(X).max())
    touched = np.zeros(1024, bool)
    touched[a0[amb0]] = True
    for g in range(1024):
        mem = a0 == g
        if not mem.any():
            assert np.array_equal(C1[g], C0[g]), g          # empty: kept bit for bit
        elif not touched[g]:
            ref = X[mem].astype(np.float64).mean(0)
            assert np.max(np.abs(C1[g] - ref)) <= 2e-6 * scale, (g, C1[g], ref)
    # the duplicate: no point goes to the higher index of the tied pair
    assert not np.any(a0 == 700) and np.array_equal(C1[700], C0[700])
    assert np.array_equal(C1[1000], C0[1000]) and np.array_equal(C1[1023], C0[1023])
    # the assignment under the returned centroids
    a1, amb1 = _nearest(X, C1)
    assert np.all((cl == a1) | amb1)
    assert np.mean(amb1) < 1e-3


def test_kmeans_warm_start_and_ties(V):
    """Two Lloyd iterations equal one iteration warm-started from one
    iteration (bit for bit); exactly tied centroids assign to the lower index."""
    X, C0 = _kmeans_case(seed=32, K=5_000)
    C2, cl2 = V.vbgs_kmeans(X, C0, 2)
    C1, _ = V.vbgs_kmeans(X, C0, 1)
    C11, cl11 = V.vbgs_kmeans(X, C1, 1)
    assert np.array_equal(C2, C11) and np.array_equal(cl2, cl11)
    # every point equidistant from two identical centroids goes to the lower one
    C = np.zeros((1024, 6), np.float32)
    C[:] = 50.0
    C[3] = C[9] = X.mean(0)
    _, cl = V.vbgs_kmeans(X, C, 0)
    assert np.all(cl == 3)
    # zero iterations only assign: centroids unchanged
    C0b, cl0 = V.vbgs_kmeans(X, C0, 0)
    assert np.array_equal(C0b, C0)
    a0, amb0 = _nearest(X, C0)
    assert np.all((cl0 == a0) | amb0)


def test_certificate_bounds_every_cluster_mass(V, room_state):
    pr, S, X2 = room_state
    K = pr["m0"].shape[0]
    m = V.Model(pr, "fp32", flags=V.VBGS_FLAG_PROPOSAL)
    m.set_stats(S)
    idx = np.random.default_rng(5).choice(X2.shape[0], 150, replace=False)
    Xs = X2[idx]
    for _ in range(3):
        ub, cl = V.vbgs_proposal_bounds(m.ctx, Xs, K)
    post = O.mstep(pr, S)
    L = O.log_rho(Xs, post)
    # the library's logits leave out -psi(sum alpha), common to all components
    shift = digamma(post["alpha"].sum()) / LN2
    sizes = np.bincount(cl, minlength=1024)
    for g in range(1024):
        if sizes[g] == 0:
            assert np.all(ub[:, g] == -np.inf)
            continue
        T = logsumexp(L[:, cl == g], axis=1) / LN2
        assert np.all(np.isfinite(ub[:, g]))
        assert np.all(ub[:, g] - shift >= T - 1e-3), (g, np.min(ub[:, g] - shift - T))
    m.close()


def test_proposal_iteration_against_exact_cavi(V, room_state):
    """One proposal iteration from the oracle's state: the certificate's
    1e-3 missed mass per point bounds the lse deficit (-ln(1 - 1e-3) nats),
    and the responsibilities' total variation per point (2e-3), hence
    sum_k |N_k - N_k^exact| <= 2e-3 N (plus FP32 rounding)."""
    pr, S, X2 = room_state
    N = X2.shape[0]
    m = V.Model(pr, "fp32", flags=V.VBGS_FLAG_PROPOSAL)
    m.set_stats(S)
    trace = m.update(X2, 1)
    rep = V.vbgs_proposal_report(m.ctx)
    assert rep["frame_exact"] == 0 and rep["fallback"] < 0.2 * N
    assert rep["audit"] > 0 and rep["audit_max_missed"] <= 1e-3
    assert rep["cand_pairs"] < 0.5 * N * S.shape[0]
    e_ref, _, lse_ref, dS_ref = O.cavi_frame(X2, pr, S, 1)
    lse = m.lse(N)
    assert np.all(lse <= lse_ref + 1e-4 * (1 + np.abs(lse_ref)))
    assert np.all(lse >= lse_ref - (-np.log1p(-1e-3)) - 1e-4 * (1 + np.abs(lse_ref)))
    assert O.relerr(trace[0], e_ref[0]) <= 1e-4
    dS = m.frame_stats()
    assert np.abs(dS[:, 0] - dS_ref[:, 0]).sum() <= 2e-3 * N + 1e-4 * N
    assert abs(dS[:, 0].sum() - N) <= 1e-3 * N
    assert O.relerr(dS[:, 1:7].sum(0), X2.sum(0)) <= 1e-3
    m.close()


def test_proposal_stream_keeps_invariants(V):
    """A short room stream with the proposal on (its first frame sees no
    surface within the depth range: an empty frame): every frame's statistics
    keep the exact totals (sum_k N_k = N, sum_k S1_k = sum_n x_n) and the
    network is trained once per non-empty frame."""
    import torch
    room = synth.Room(seed=22)
    pr = synth.room_prior(20_000, seed=22)
    m = V.Model(pr, "fp32", flags=V.VBGS_FLAG_PROPOSAL)
    trained = 0
    sizes = []
    for t in range(4):
        X = synth.room_frame(t, seed=22, width=120, height=120, room=room)
        sizes.append(X.shape[0])
        tr = m.update(torch.from_numpy(X).cuda(), 3)
        assert np.all(np.isfinite(tr))
        rep = V.vbgs_proposal_report(m.ctx)
        if X.shape[0] == 0:
            assert np.all(m.frame_stats() == 0)
            continue
        trained += 1
        dS = m.frame_stats()
        assert abs(dS[:, 0].sum() - X.shape[0]) <= 1e-3 * X.shape[0]
        assert O.relerr(dS[:, 1:7].sum(0), X.sum(0)) <= 1e-3
        assert rep["frames_trained"] == trained
        assert rep["points"] == X.shape[0]
        assert rep["audit_max_missed"] <= 1e-3
    assert sizes[0] == 0 and trained >= 2
    m.close()


def test_trained_network_needs_fewer_candidates(V):
    """The ablation of the learned part: one room stream (K = 20,000, 120 x 120
    frames, FP16x3 exact E-step) with the network trained online on the exact
    E-steps' cluster masses (the default schedule) and with the same network
    frozen at its initial weights, under the same certificate expansion.
    Over frames 24-35 the trained network's top-4 leaves less for the
    certificate to add: fewer candidate pairs and fewer added clusters per
    point, with the audit's true missed mass within 1e-3 in both runs."""
    import torch
    K = 20_000
    pr = synth.room_prior(K, seed=5)
    room = synth.Room(5)
    frames = [torch.from_numpy(synth.room_frame(t, seed=5, width=120, height=120, room=room)).cuda()
              for t in range(36)]
    out = {}
    for name, epochs in (("trained", 8), ("frozen", 0)):
        m = V.Model(pr, "fp16x3", flags=V.VBGS_FLAG_PROPOSAL)
        V.vbgs_proposal_config(m.ctx, epochs, 3e-3)
        pairs = added = pts = 0.0
        for t, X in enumerate(frames):
            m.update(X, 3)
            r = V.vbgs_proposal_report(m.ctx)
            assert r["audit_max_missed"] <= 1e-3
            if t >= 24 and not r["frame_exact"]:
                pairs += r["cand_pairs"]
                added += r["added_clusters"]
                pts += r["points"]
        out[name] = (pairs / (pts * K), added / pts, r["train_loss"])
        m.close()
    print(f"\nablation (candidate pair fraction, clusters added per point, last loss): {out}")
    assert out["trained"][0] <= 0.9 * out["frozen"][0], out
    assert out["trained"][1] <= 0.8 * out["frozen"][1], out
