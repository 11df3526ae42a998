"""GPU parity of the splat renderer and PSNR (vbgs_render) with the oracle's
renderer (oracle/render.py) on held-out views of the room stream.

The posterior comes from the FP64 oracle's own CAVI frames (set into the
context with vbgs_set_stats); the camera is a pose of the stream that no
frame was lifted from.  The renderer evaluates alpha in FP32, the oracle in
FP64, and a splat is skipped where alpha < 1/255: a (splat, pixel) pair
whose alpha lies at that threshold may be kept on one side and skipped on
the other.  Such a pair changes the pixel by at most 2/255 (its own
contribution, alpha <= 1/255 of a colour <= 1, and the same factor on the
transmittance of the splats behind it), so the per-pixel bound is the FP32
rounding of the compositing, 2e-6 + 4e-7 per contributing splat (each step
rounds alpha, the transmittance and the colour sums: a few units of 2^-24
each, and ex2.approx two), plus 2/255 per threshold pair of the pixel, the
pairs found in FP64 (|q - q_min| <= 1e-5 q_min: fifty times the FP32 error
of q).  Such pixels are rare (checked), and the PSNR must agree
to 0.01 dB.  For the oracle's image of a large view, splats whose alpha
region lies outside the image (checked in FP64 with a margin) are left out
of its input: they add nothing to any pixel, so its result is unchanged.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from oracle import render as RD
from oracle import split as SP
from paper_2603_08499_gb300 import synth

pytestmark = pytest.mark.gpu

Q_MIN = 2.0 * np.log(255.0 * 0.99)     # alpha >= 1/255  <=>  q <= Q_MIN


@pytest.fixture(scope="module")
def V():
    from paper_2603_08499_gb300 import build
    build.build()
    from paper_2603_08499_gb300 import vbgs
    return vbgs


def threshold_pairs(mu, Sigma, cam):
    """Per pixel: the number of splats whose FP64 q lies at the alpha
    threshold, and the number of splats that contribute (alpha >= 1/255)."""
    uv, z, C = RD.project(mu, Sigma, cam)
    W, H = cam["width"], cam["height"]
    count = np.zeros((H, W), dtype=np.int64)
    contrib = np.zeros((H, W), dtype=np.int64)
    for k in np.flatnonzero(z > RD.NEAR):
        hx, hy = np.sqrt(Q_MIN * C[k, 0, 0]) * 1.01 + 1, np.sqrt(Q_MIN * C[k, 1, 1]) * 1.01 + 1
        i0, i1 = max(int(np.floor(uv[k, 0] - hx)), 0), min(int(np.ceil(uv[k, 0] + hx)), W - 1)
        j0, j1 = max(int(np.floor(uv[k, 1] - hy)), 0), min(int(np.ceil(uv[k, 1] + hy)), H - 1)
        if i0 > i1 or j0 > j1:
            continue
        pu, pv = np.meshgrid(np.arange(i0, i1 + 1) + 0.5, np.arange(j0, j1 + 1) + 0.5)
        d = np.stack([pu - uv[k, 0], pv - uv[k, 1]], axis=-1)
        q = np.einsum("...i,ij,...j->...", d, np.linalg.inv(C[k]), d)
        count[j0:j1 + 1, i0:i1 + 1] += np.abs(q - Q_MIN) <= 1e-5 * Q_MIN
        contrib[j0:j1 + 1, i0:i1 + 1] += q <= Q_MIN
    return count, contrib


def on_image(mu, Sigma, cam):
    """Splats in front of the camera whose alpha >= 1/255 region (with a
    margin) meets the image."""
    uv, z, C = RD.project(mu, Sigma, cam)
    hx = np.sqrt(Q_MIN * np.abs(C[:, 0, 0])) * 1.01 + 2
    hy = np.sqrt(Q_MIN * np.abs(C[:, 1, 1])) * 1.01 + 2
    return (z > RD.NEAR) & (uv[:, 0] + hx >= 0) & (uv[:, 0] - hx <= cam["width"]) & \
        (uv[:, 1] + hy >= 0) & (uv[:, 1] - hy <= cam["height"])


def check_image(img, ref_img, counts):
    pairs, contrib = counts
    err = np.abs(img.astype(np.float64) - ref_img).max(axis=2)
    fp32 = 2e-6 + 4e-7 * contrib
    allowed = fp32 + pairs * (2.0 / 255.0) * 1.01
    assert np.all(err <= allowed), (float(err.max()), int(np.sum(err > allowed)))
    assert np.mean(pairs > 0) < 0.05
    return float(np.max(np.where(pairs == 0, err / fp32, 0.0)))


def fitted_state(seed, K, n_frames, w, iters):
    room = synth.Room(seed)
    pr = synth.room_prior(K, seed=seed)
    S = np.zeros((K, 28))
    for t in range(n_frames):
        X = synth.room_frame(t, seed=seed, width=w, height=w, room=room)
        S = O.cavi_frame(X, pr, S, iters)[1]
    return room, pr, S


@pytest.mark.parametrize("pose", [100, 101])
def test_render_matches_oracle_small(V, pose):
    room, pr, S = fitted_state(51, 3_000, 3, 64, 3)
    view = synth.room_view(pose, seed=51, width=96, height=80, room=room)
    post = O.mstep(pr, S)
    ref = RD.render_posterior(post, view, S[:, 0])
    m = V.Model(pr, "fp64")
    m.set_stats(S)
    img, p, ms = m.render(view, reference=view["image"])
    m.close()
    assert img.shape == (80, 96, 3) and ms > 0
    k = RD.drawn(S[:, 0])
    err = check_image(img, ref, threshold_pairs(post["m"][k, :3],
                                                RD.expected_spatial_cov(post["Winv"][k], post["nu"][k], 6), view))
    assert err <= 1.0
    assert abs(p - RD.psnr(ref, view["image"])) <= 0.01
    assert np.any(img > 0.05)


def test_render_full_size_against_oracle(V):
    """K = 50,000 components, a 200 x 200 held-out view (the benchmark's
    resolution and component count)."""
    room, pr, S = fitted_state(2, 50_000, 2, 200, 1)
    view = synth.room_view(1000, seed=2, room=room)
    post = O.mstep(pr, S)
    mu, Sigma = post["m"][:, :3], RD.expected_spatial_cov(post["Winv"], post["nu"], 6)
    keep = on_image(mu, Sigma, view) & (S[:, 0] >= RD.MIN_COUNT)
    ref = RD.render(mu[keep], Sigma[keep], post["m"][keep, 3:], view)
    m = V.Model(pr, "fp16x3")
    m.set_stats(S)
    img, p, _ = m.render(view, reference=view["image"])
    m.close()
    check_image(img, ref, threshold_pairs(mu[keep], Sigma[keep], view))
    assert abs(p - RD.psnr(ref, view["image"])) <= 0.01


def test_render_split_model(V):
    """The split model's spatial block (d = 3) against the split oracle."""
    room = synth.Room(52)
    pr = synth.room_prior(2_000, seed=52)
    S = np.zeros((2_000, 28))
    for t in range(2):
        S = SP.cavi_frame(synth.room_frame(t, seed=52, width=64, height=64, room=room), pr, S, 2)[1]
    view = synth.room_view(77, seed=52, width=64, height=64, room=room)
    qs, qc = SP.mstep(pr, S)
    k = RD.drawn(S[:, 0])
    mu, Sigma = qs["m"][k], RD.expected_spatial_cov(qs["Winv"][k], qs["nu"][k], 3)
    ref = RD.render(mu, Sigma, qc["m"][k], view)
    m = V.Model(pr, "fp64", flags=V.VBGS_FLAG_SPLIT)
    m.set_stats(S)
    img, p, _ = m.render(view, reference=view["image"])
    m.close()
    check_image(img, ref, threshold_pairs(mu, Sigma, view))
    assert abs(p - RD.psnr(ref, view["image"])) <= 0.01


def test_render_edges(V):
    _, pr = synth.c1_workload(seed=53, N=10, K=50)
    m = V.Model(pr, "fp64")
    # looking away from every splat: a black image, infinite PSNR against black
    cam = {"o": np.array([0.0, 0.0, 50.0]), "Rwc": np.eye(3), "f": 40.0, "width": 33, "height": 17}
    img, p, _ = m.render(cam, reference=np.zeros((17, 33, 3)))
    assert np.all(img == 0) and p == np.inf
    # a model no data has reached draws nothing
    cam = {"o": np.array([0.0, 0.0, -3.0]), "Rwc": np.eye(3), "f": 20.0, "width": 37, "height": 19}
    img, _, _ = m.render(cam)
    assert np.all(img == 0)
    # a 1 x 1 image and a ragged tile grid against the oracle; every third
    # component without data (not drawn)
    X, _ = synth.c1_workload(seed=53, N=3_000, K=50)
    S = O.cavi_frame(X, pr, np.zeros((50, 28)), 3)[1]
    S[::3] = 0.0
    m.set_stats(S)
    post = O.mstep(pr, S)
    k = RD.drawn(S[:, 0])
    assert 0 < k.size < 50
    for W, H in ((1, 1), (37, 19)):
        cam = {"o": np.array([0.0, 0.0, -3.0]), "Rwc": np.eye(3), "f": 20.0, "width": W, "height": H}
        img, _, _ = m.render(cam)
        ref = RD.render_posterior(post, cam, S[:, 0])
        check_image(img, ref, threshold_pairs(post["m"][k, :3],
                                              RD.expected_spatial_cov(post["Winv"][k], post["nu"][k], 6), cam))
    for bad in ({"width": 0}, {"f": -1.0}):
        c = dict(cam, **bad)
        with pytest.raises((V.VbgsError, ValueError)):
            m.render(c)
    # a PSNR without a reference image
    rc = V.lib().vbgs_render(m.ctx, V._dp(V.camera_array(cam)), 4, 4, None, None, V._dp(np.zeros(1)), None)
    assert rc == V.VBGS_EINVAL
    m.close()
