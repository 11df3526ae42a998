"""Pins of the oracle's splat renderer and PSNR (CPU only) against results
other than itself: an isotropic splat's image against its closed form, the
EWA screen covariance against the covariance of exactly projected samples,
the expected covariance of a Wishart posterior against sampled inverses, the
compositing order, splats behind the camera, and PSNR's closed forms.  A
wrong Jacobian sign or scale, a missing low-pass, a wrong (nu - d - 1), a
back-to-front order or a PSNR on the wrong scale fails one of them."""
from __future__ import annotations

import numpy as np
from scipy import stats
from scipy.spatial.transform import Rotation

from oracle import render as RD


def _cam(W=41, H=41, f=50.0, Rwc=None, o=None):
    return {"o": np.zeros(3) if o is None else o, "Rwc": np.eye(3) if Rwc is None else Rwc, "f": f,
            "width": W, "height": H}


def test_isotropic_splat_profile_is_the_closed_form():
    cam = _cam()
    s, z = 0.05, 2.0
    img = RD.render(np.array([[0.0, 0.0, z]]), np.array([np.eye(3) * s * s]), np.array([[1.0, 0.25, 0.0]]), cam,
                    opacity=0.9)
    var = (cam["f"] * s / z) ** 2 + 0.3
    i = np.arange(41)
    d2 = (i - 20.0) ** 2
    a = 0.9 * np.exp(-0.5 * d2 / var)
    a = np.where(a >= 1 / 255, a, 0.0)
    assert np.allclose(img[20, :, 0], a, rtol=0, atol=1e-12)          # the row through the centre
    assert np.allclose(img[:, 20, 1], 0.25 * a, rtol=0, atol=1e-12)   # the column, green channel
    assert np.all(img[..., 2] == 0.0)


def test_screen_covariance_is_that_of_projected_samples():
    rng = np.random.default_rng(31)
    Rwc = Rotation.from_euler("xyz", [0.2, -0.3, 0.1]).as_matrix()
    cam = _cam(W=200, H=160, f=120.0, Rwc=Rwc, o=np.array([0.1, -0.2, 0.3]))
    A = rng.standard_normal((3, 3))
    Sigma = (A @ A.T + 0.5 * np.eye(3)) * 1e-4
    xc_mean = np.array([0.35, -0.25, 2.5])
    mu = cam["o"] + Rwc @ xc_mean
    uv, z, C = RD.project(mu[None, :], Sigma[None, :, :], cam)
    X = rng.multivariate_normal(mu, Sigma, size=200_000)
    xc = (X - cam["o"]) @ Rwc                      # world -> camera: Rcw = Rwc^T
    p = np.stack([cam["f"] * xc[:, 0] / xc[:, 2], cam["f"] * xc[:, 1] / xc[:, 2]], axis=1)
    emp = np.cov(p.T)
    assert abs(z[0] - 2.5) < 1e-12
    assert np.allclose(uv[0], [cam["f"] * 0.35 / 2.5 + 100.0, cam["f"] * -0.25 / 2.5 + 80.0], atol=1e-9)
    assert np.allclose(C[0] - 0.3 * np.eye(2), emp, rtol=0.02, atol=0.02 * np.abs(emp).max())


def test_expected_covariance_of_a_wishart_posterior():
    rng = np.random.default_rng(32)
    for d, nu in ((3, 9.0), (6, 12.0)):
        A = rng.standard_normal((d, d))
        Winv = A @ A.T + np.eye(d)
        Lam = stats.wishart(df=nu, scale=np.linalg.inv(Winv)).rvs(size=100_000, random_state=rng)
        mc = np.linalg.inv(Lam).mean(axis=0)[:3, :3]
        ref = RD.expected_spatial_cov(Winv[None], np.array([nu]), d)[0]
        assert np.allclose(mc, ref, rtol=0.03, atol=0.03 * np.abs(ref).max()), (d, mc, ref)


def test_compositing_is_front_to_back_whatever_the_input_order():
    cam = _cam()
    mu = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 2.0]])
    S = np.array([np.eye(3) * 0.02 ** 2, np.eye(3) * 0.04 ** 2])
    col = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    a = RD.render(mu, S, col, cam)
    b = RD.render(mu[::-1], S[::-1], col[::-1], cam)
    assert np.array_equal(a, b)
    # at the centre both splats have alpha 0.99: red 0.99, blue 0.99 * 0.01
    assert np.allclose(a[20, 20], [0.99, 0.0, 0.99 * 0.01], atol=1e-12)


def test_splats_behind_or_at_the_camera_are_left_out():
    cam = _cam()
    S = np.array([np.eye(3) * 0.1 ** 2] * 2)
    img = RD.render(np.array([[0.0, 0.0, -1.0], [0.0, 0.0, 0.05]]), S, np.ones((2, 3)), cam)
    assert np.all(img == 0.0)


def test_psnr_closed_forms():
    rng = np.random.default_rng(33)
    a = rng.random((8, 9, 3))
    assert RD.psnr(a, a) == float("inf")
    assert abs(RD.psnr(a, a + 0.1) - 20.0) < 1e-9                       # -20 log10(0.1)
    assert abs(RD.psnr(a, a - 1 / 255) - 20 * np.log10(255.0)) < 1e-9   # one grey level everywhere


def test_only_components_with_data_are_drawn():
    """render_posterior draws exactly the components whose accumulated count
    is at least one point: one below (0.999) leaves the image as without it,
    one at 1.0 changes it; the posterior's own values are used unchanged."""
    cam = _cam()
    K = 3
    post = {"m": np.array([[0.0, 0.0, 2.0, 1.0, 0.0, 0.0], [0.05, 0.0, 2.5, 0.0, 1.0, 0.0],
                           [-0.05, 0.0, 3.0, 0.0, 0.0, 1.0]]),
            "Winv": np.array([np.eye(6) * 0.01 * (i + 1) for i in range(K)]), "nu": np.full(K, 12.0)}
    full = RD.render_posterior(post, cam, np.array([5.0, 1.0, 2.0]))
    cov = RD.expected_spatial_cov(post["Winv"], post["nu"], 6)
    assert np.array_equal(full, RD.render(post["m"][:, :3], cov, post["m"][:, 3:], cam))
    part = RD.render_posterior(post, cam, np.array([5.0, 0.999, 2.0]))
    keep = [0, 2]
    assert np.array_equal(part, RD.render(post["m"][keep, :3], cov[keep], post["m"][keep, 3:], cam))
    assert not np.allclose(part, full)
    assert np.all(RD.render_posterior(post, cam, np.zeros(K)) == 0.0)
