"""Seeded synthetic inputs for the VBGS update: point clouds and priors.

This module draws data only; it holds none of the update's arithmetic, so
both the CUDA path and the FP64 oracle can take their inputs from it.  The
generated shapes stand in for the paper's RGB-D datasets (Blender, Habitat,
Replica), which are not used:

* ``mixture_points``: joint 6-D points (xyz in [-1, 1]^3, rgb in [0, 1]^3)
  from a ground-truth mixture of anisotropic Gaussians with random rotations
  and axis scales, uniform per-point colours, plus uniform outliers.
* ``room_frame``: one lifted RGB-D frame of a procedurally textured box room
  with ellipsoids, seen by a pinhole camera from a random pose (depth
  clipped to [0.5, 5] m; colour per 0.5 m surface patch plus N(0, 0.02)
  noise).  Frames of one stream share the room and differ in pose.
* ``nw_prior``: the Normal-Wishart / Dirichlet prior of K components with
  means m0 drawn uniformly in a box.
"""
from __future__ import annotations

import math

import numpy as np


def _rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random 3x3 rotation: QR of a Gaussian matrix with a sign fix."""
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def mixture_points(N: int = 10_000, n_gauss: int = 50, seed: int = 1, outlier_frac: float = 0.05,
                   scale_lo: float = 0.02, scale_hi: float = 0.2) -> np.ndarray:
    """N x 6 float64 points: (1 - outlier_frac) N from the Gaussian mixture,
    the rest uniform in [-1, 1]^3 x [0, 1]^3; rows shuffled."""
    rng = np.random.default_rng(seed)
    n_out = int(round(outlier_frac * N))
    n_in = N - n_out
    centers = rng.uniform(-1.0, 1.0, (n_gauss, 3))
    rots = np.stack([_rotation(rng) for _ in range(n_gauss)])
    scales = rng.uniform(scale_lo, scale_hi, (n_gauss, 3))
    lab = rng.integers(0, n_gauss, n_in)
    z = rng.standard_normal((n_in, 3)) * scales[lab]
    pos = centers[lab] + np.einsum("nij,nj->ni", rots[lab], z)
    col = rng.uniform(0.0, 1.0, (n_in, 3))
    out = np.concatenate([rng.uniform(-1.0, 1.0, (n_out, 3)), rng.uniform(0.0, 1.0, (n_out, 3))], axis=1)
    X = np.concatenate([np.concatenate([pos, col], axis=1), out], axis=0)
    return np.ascontiguousarray(X[rng.permutation(N)])


def nw_prior(K: int, seed: int, lo=(-1, -1, -1, 0, 0, 0), hi=(1, 1, 1, 1, 1, 1), alpha0: float = 1.0,
             beta0: float = 1.0, nu0: float = 8.0, w0_scale: float = 100.0) -> dict:
    """Prior of K components: m0 uniform in the box [lo, hi], W0 = w0_scale I
    (precision space, i.e. prior scale 1/sqrt(w0_scale) per axis)."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    m0 = lo + (hi - lo) * rng.uniform(size=(K, 6))
    return {"alpha0": float(alpha0), "beta0": float(beta0), "nu0": float(nu0),
            "m0": np.ascontiguousarray(m0), "W0": np.eye(6) * float(w0_scale)}


# ---- procedural room ---------------------------------------------------------

ROOM_LO = np.array([-3.0, -3.0, 0.0])
ROOM_HI = np.array([3.0, 3.0, 3.0])
PATCH = 0.5


class Room:
    """A 6 x 6 x 3 m box room with 6 ellipsoids; seeded, deterministic."""

    def __init__(self, seed: int = 2, n_ellipsoids: int = 6):
        rng = np.random.default_rng([seed, 7919])
        n_patch = int(round(6.0 / PATCH))
        # one colour table per box face (6 faces), indexed by patch (u, v)
        self.face_colors = rng.uniform(0.0, 1.0, (6, n_patch, n_patch, 3))
        self.ell_center = np.stack([rng.uniform(-2.0, 2.0, n_ellipsoids), rng.uniform(-2.0, 2.0, n_ellipsoids),
                                    rng.uniform(0.4, 2.2, n_ellipsoids)], axis=1)
        self.ell_axes = rng.uniform(0.2, 0.7, (n_ellipsoids, 3))
        self.ell_rot = np.stack([_rotation(rng) for _ in range(n_ellipsoids)])
        # ellipsoid surface patches: 8 octants, one colour each
        self.ell_colors = rng.uniform(0.0, 1.0, (n_ellipsoids, 8, 3))

    def cast(self, o: np.ndarray, d: np.ndarray):
        """Nearest hit of rays o + t d (d: R x 3).  Returns t (R,), colour (R x 3)."""
        R = d.shape[0]
        t_best = np.full(R, np.inf)
        col = np.zeros((R, 3))
        # box interior: exit distance through each face plane
        with np.errstate(divide="ignore", invalid="ignore"):
            for axis in range(3):
                for side, bound in ((0, ROOM_LO[axis]), (1, ROOM_HI[axis])):
                    t = (bound - o[axis]) / d[:, axis]
                    ok = (t > 1e-9) & (t < t_best)
                    if not ok.any():
                        continue
                    p = o[None, :] + t[:, None] * d
                    other = [a for a in range(3) if a != axis]
                    inside = np.all((p[:, other] >= ROOM_LO[other] - 1e-9) & (p[:, other] <= ROOM_HI[other] + 1e-9), axis=1)
                    ok &= inside
                    face = 2 * axis + side
                    u = np.clip(((p[:, other[0]] - ROOM_LO[other[0]]) / PATCH).astype(int), 0, self.face_colors.shape[1] - 1)
                    v = np.clip(((p[:, other[1]] - ROOM_LO[other[1]]) / PATCH).astype(int), 0, self.face_colors.shape[2] - 1)
                    t_best = np.where(ok, t, t_best)
                    col[ok] = self.face_colors[face, u[ok], v[ok]]
        for e in range(self.ell_center.shape[0]):
            Rm, ax, c = self.ell_rot[e], self.ell_axes[e], self.ell_center[e]
            # ray in the ellipsoid's unit-sphere frame
            oo = (Rm.T @ (o - c)) / ax
            dd = (d @ Rm) / ax
            a = np.sum(dd * dd, axis=1)
            b = 2.0 * (dd @ oo)
            cc = oo @ oo - 1.0
            disc = b * b - 4 * a * cc
            hit = disc > 0
            sq = np.sqrt(np.where(hit, disc, 0.0))
            t0 = (-b - sq) / (2 * a)
            t1 = (-b + sq) / (2 * a)
            t = np.where(t0 > 1e-9, t0, t1)
            ok = hit & (t > 1e-9) & (t < t_best)
            if ok.any():
                p_local = oo[None, :] + t[:, None] * dd
                octant = (p_local[:, 0] > 0).astype(int) + 2 * (p_local[:, 1] > 0) + 4 * (p_local[:, 2] > 0)
                t_best = np.where(ok, t, t_best)
                col[ok] = self.ell_colors[e, octant[ok]]
        return t_best, col


def camera_pose(rng: np.random.Generator):
    """Random camera inside the room looking at a random target: (origin, R_world_from_cam)."""
    o = np.array([rng.uniform(-2.5, 2.5), rng.uniform(-2.5, 2.5), rng.uniform(0.5, 2.5)])
    while True:
        tgt = np.array([rng.uniform(-3, 3), rng.uniform(-3, 3), rng.uniform(0, 3)])
        fwd = tgt - o
        if np.linalg.norm(fwd) > 1.0:
            break
    fwd /= np.linalg.norm(fwd)
    up = np.array([0.0, 0.0, 1.0])
    right = np.cross(fwd, up)
    if np.linalg.norm(right) < 1e-6:
        right = np.array([1.0, 0.0, 0.0])
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    return o, np.stack([right, down, fwd], axis=1)   # columns: camera x, y, z axes in world


def room_frame(t: int, seed: int = 2, width: int = 200, height: int = 200, fov_deg: float = 60.0,
               dmin: float = 0.5, dmax: float = 5.0, color_noise: float = 0.02, room: Room | None = None) -> np.ndarray:
    """Frame t of the seeded room stream: N x 6 float64 lifted RGB-D points
    (world xyz in metres, rgb in [0, 1]); N <= width * height after the
    depth clip."""
    room = room or Room(seed)
    rng = np.random.default_rng([seed, t])
    o, Rwc = camera_pose(rng)
    f = (width / 2.0) / math.tan(math.radians(fov_deg) / 2.0)
    u, v = np.meshgrid(np.arange(width) + 0.5, np.arange(height) + 0.5)
    dirs_cam = np.stack([(u.ravel() - width / 2.0) / f, (v.ravel() - height / 2.0) / f, np.ones(u.size)], axis=1)
    dirs = dirs_cam @ Rwc.T
    tt, col = room.cast(o, dirs)
    depth = tt   # z-depth along the optical axis (dirs_cam has unit z)
    keep = np.isfinite(depth) & (depth >= dmin) & (depth <= dmax)
    pts = o[None, :] + tt[keep, None] * dirs[keep]
    c = np.clip(col[keep] + rng.normal(0.0, color_noise, (int(keep.sum()), 3)), 0.0, 1.0)
    return np.ascontiguousarray(np.concatenate([pts, c], axis=1))


def room_view(t: int, seed: int = 2, width: int = 200, height: int = 200, fov_deg: float = 60.0,
              dmin: float = 0.5, dmax: float = 5.0, room: Room | None = None) -> dict:
    """The pinhole view of pose t of the seeded room stream as an image (the
    ground truth of a held-out view): camera centre o, camera-to-world
    rotation Rwc, focal length f (pixels), the colour image (height x width x
    3 in [0, 1], no noise; 0 where nothing lies within [dmin, dmax]) and its
    hit mask.  Pixel (u, v) looks along Rwc ((u + 1/2 - width/2) / f,
    (v + 1/2 - height/2) / f, 1), as in room_frame."""
    room = room or Room(seed)
    rng = np.random.default_rng([seed, t])
    o, Rwc = camera_pose(rng)
    f = (width / 2.0) / math.tan(math.radians(fov_deg) / 2.0)
    u, v = np.meshgrid(np.arange(width) + 0.5, np.arange(height) + 0.5)
    dirs_cam = np.stack([(u.ravel() - width / 2.0) / f, (v.ravel() - height / 2.0) / f, np.ones(u.size)], axis=1)
    tt, col = room.cast(o, dirs_cam @ Rwc.T)
    hit = np.isfinite(tt) & (tt >= dmin) & (tt <= dmax)
    img = np.where(hit[:, None], col, 0.0).reshape(height, width, 3)
    return {"o": o, "Rwc": Rwc, "f": f, "width": width, "height": height, "image": img,
            "mask": hit.reshape(height, width)}


def room_prior(K: int, seed: int = 2, **kw) -> dict:
    """Prior for the room stream: m0 uniform in the room box x [0, 1]^3."""
    return nw_prior(K, seed=seed + 1000, lo=tuple(ROOM_LO) + (0, 0, 0), hi=tuple(ROOM_HI) + (1, 1, 1), **kw)


def c1_workload(seed: int = 1, N: int = 10_000, K: int = 1_000):
    """Plain FP64 VBGS update workload: mixture points + prior of K components."""
    return mixture_points(N=N, seed=seed), nw_prior(K, seed=seed + 100)


def scene_sizes(n_scenes: int = 64, seed: int = 4, n_lo=5_000, n_hi=160_000, k_lo=1_000, k_hi=50_000):
    """(N, K) of uneven scenes, both log-uniform."""
    rng = np.random.default_rng(seed)
    N = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), n_scenes)).astype(np.int64)
    K = np.exp(rng.uniform(math.log(k_lo), math.log(k_hi), n_scenes)).astype(np.int64)
    return N, K
