"""Splat rendering of a fitted mixture and the PSNR of Sec. 5.1 --
TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline /
reference legs may import this module.  It shares no code with the CUDA
library.

The paper measures reconstruction quality as PSNR = 10 log10(255^2 / MSE)
on held-out views, MSE the mean over all pixels and RGB channels of the
squared differences of the two images on a 0..255 scale (Sec. 5.1); it does
not describe how the mixture is rendered.  Readings (each stated in the
design notes):

* every component that data has reached -- accumulated count N_k >= 1, at
  least one point's worth of responsibility -- is a splat; the others hold
  only the prior, which says nothing about the scene, and are left out;
* a splat sits at its spatial posterior mean m_s with the
  expected spatial covariance E[Sigma_s] = W_s^-1 / (nu - d - 1) of its
  Wishart posterior (d = 6 for the joint model, taking the spatial block of
  W^-1; d = 3 for the split model's spatial block), its colour the colour
  posterior mean clamped to [0, 1], its opacity a constant o (0.99);
* projection as elliptical weighted average splatting (Zwicker et al. 2001):
  camera-space mean x_c, the perspective Jacobian J at x_c, screen covariance
  J R Sigma R^T J^T plus 0.3 px^2 on its diagonal (the screen-space low-pass);
  splats closer than 0.1 m to the camera plane are left out;
* front-to-back compositing at each pixel centre, in increasing camera depth
  (ties by component index): alpha_k = min(0.99, o exp(-1/2 d^T C_k^-1 d)),
  colour += T alpha_k c_k, T *= 1 - alpha_k, contributions with alpha below
  1/255 skipped; the background (black) takes the remaining T.
The camera follows synth.room_view: pixel (u, v) looks along
Rwc ((u + 1/2 - width/2) / f, (v + 1/2 - height/2) / f, 1) from o.

Pins: tests/test_render_pins.py (an isotropic splat's profile against its
closed form, the Jacobian's screen covariance against projected Monte Carlo
samples, the expected covariance against sampled Wishart inverses, the
compositing order, splats behind the camera, and PSNR's closed forms).
"""
from __future__ import annotations

import numpy as np

NEAR = 0.1
LOW_PASS = 0.3
MIN_COUNT = 1.0
ALPHA_MAX = 0.99
ALPHA_MIN = 1.0 / 255.0


def expected_spatial_cov(Winv, nu, d: int) -> np.ndarray:
    """E[Sigma] of the spatial block: W^-1[:3, :3] / (nu - d - 1), K x 3 x 3."""
    Winv = np.asarray(Winv, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    return Winv[:, :3, :3] / (nu - d - 1.0)[:, None, None]


def project(mu, Sigma, cam: dict):
    """(pixel centres K x 2, depths K, screen covariances K x 2 x 2) of splats
    with world means mu (K x 3) and covariances Sigma (K x 3 x 3)."""
    Rcw = np.asarray(cam["Rwc"], dtype=np.float64).T
    xc = (np.asarray(mu, dtype=np.float64) - np.asarray(cam["o"])[None, :]) @ Rcw.T
    f, W, H = cam["f"], cam["width"], cam["height"]
    z = xc[:, 2]
    zs = np.where(z > NEAR, z, 1.0)
    uv = np.stack([f * xc[:, 0] / zs + W / 2.0, f * xc[:, 1] / zs + H / 2.0], axis=1)
    J = np.zeros((xc.shape[0], 2, 3))
    J[:, 0, 0] = f / zs
    J[:, 0, 2] = -f * xc[:, 0] / zs ** 2
    J[:, 1, 1] = f / zs
    J[:, 1, 2] = -f * xc[:, 1] / zs ** 2
    Sc = Rcw[None, :, :] @ np.asarray(Sigma, dtype=np.float64) @ Rcw.T[None, :, :]
    C = J @ Sc @ np.transpose(J, (0, 2, 1)) + LOW_PASS * np.eye(2)[None, :, :]
    return uv, z, C


def render(mu, Sigma, colour, cam: dict, opacity: float = ALPHA_MAX) -> np.ndarray:
    """The height x width x 3 image of the splats (front to back, black
    background)."""
    uv, z, C = project(mu, Sigma, cam)
    colour = np.clip(np.asarray(colour, dtype=np.float64), 0.0, 1.0)
    keep = np.flatnonzero(z > NEAR)
    order = keep[np.lexsort((keep, z[keep]))]           # increasing depth, ties by index
    Ci = np.linalg.inv(C[order])
    W, H = cam["width"], cam["height"]
    pu, pv = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    px = np.stack([pu.ravel(), pv.ravel()], axis=1)      # P x 2
    out = np.zeros((px.shape[0], 3))
    T = np.ones(px.shape[0])
    for i, k in enumerate(order):
        d = px - uv[k][None, :]
        q = np.einsum("pi,ij,pj->p", d, Ci[i], d)
        a = np.minimum(ALPHA_MAX, opacity * np.exp(-0.5 * q))
        a = np.where(a >= ALPHA_MIN, a, 0.0)
        out += (T * a)[:, None] * colour[k][None, :]
        T *= 1.0 - a
    return out.reshape(H, W, 3)


def drawn(counts) -> np.ndarray:
    """Indices of the components that are splats: accumulated count >= 1."""
    return np.flatnonzero(np.asarray(counts, dtype=np.float64) >= MIN_COUNT)


def render_posterior(post: dict, cam: dict, counts, d: int = 6, opacity: float = ALPHA_MAX) -> np.ndarray:
    """Render a joint posterior (m K x 6, Winv K x 6 x 6, nu K) whose
    components have accumulated the counts N_k (K)."""
    k = drawn(counts)
    m = np.asarray(post["m"], dtype=np.float64)[k]
    return render(m[:, :3], expected_spatial_cov(np.asarray(post["Winv"])[k], np.asarray(post["nu"])[k], d),
                  m[:, 3:], cam, opacity)


def psnr(img, ref) -> float:
    """10 log10(255^2 / MSE), images in [0, 1] put on the 0..255 scale."""
    diff = 255.0 * (np.asarray(img, dtype=np.float64) - np.asarray(ref, dtype=np.float64))
    mse = float(np.mean(diff * diff))
    return float("inf") if mse == 0.0 else 10.0 * np.log10(255.0 ** 2 / mse)
