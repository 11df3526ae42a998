"""The input generator's ground-truth views (CPU only): for a pose of the
room stream, the pixels the view marks as hits are exactly the points
room_frame lifts for that pose (same count, the points on the pixels' rays),
and their colours are the frame's colours before its N(0, 0.02) noise."""
from __future__ import annotations

import numpy as np

from paper_2603_08499_gb300 import synth


def test_room_view_matches_the_lifted_frame_of_the_same_pose():
    room = synth.Room(seed=3)
    W, H = 48, 40
    for t in (0, 5):
        X = synth.room_frame(t, seed=3, width=W, height=H, room=room)
        v = synth.room_view(t, seed=3, width=W, height=H, room=room)
        assert v["image"].shape == (H, W, 3) and v["mask"].sum() == X.shape[0]
        # project the lifted points back into the view: each lands on its own hit pixel
        xc = (X[:, :3] - v["o"]) @ v["Rwc"]
        u = v["f"] * xc[:, 0] / xc[:, 2] + W / 2.0
        w = v["f"] * xc[:, 1] / xc[:, 2] + H / 2.0
        iu, iv = np.floor(u).astype(int), np.floor(w).astype(int)
        assert np.allclose(u - iu, 0.5, atol=1e-6) and np.allclose(w - iv, 0.5, atol=1e-6)
        assert np.all(v["mask"][iv, iu])
        # colours: the view's noise-free colour within 5 sigma of the frame's noise (clamped to [0, 1])
        d = X[:, 3:] - v["image"][iv, iu]
        assert np.all(np.abs(d) <= 5 * 0.02 + 1e-12)
        assert abs(d.mean()) < 0.01
        assert np.all(v["image"][~v["mask"]] == 0.0)
