"""GPU tests of the continual state and the context options through the C ABI.

* vbgs_save_state / vbgs_load_state (Alg. 1's model and statistics buffer
  carried across frames, Sec. 2.1.2): a stream saved after k frames, its
  context destroyed and the file loaded into a new context, continues bit
  for bit like the uninterrupted stream -- ELBO traces, statistics,
  posterior, lse and, with the learned proposal, the network's weights.
* A damaged, truncated or missing state file is refused (VBGS_EIO).
* options.checks: the frame consistency checks change no result, and the
  check kernel flags non-finite, negative and non-conserved statistics.
* options.seed and options.autotune_cache.
"""
from __future__ import annotations

import os

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


def _frames(seed, n, w=120, h=120):
    import torch
    room = synth.Room(seed=seed)
    return [torch.from_numpy(synth.room_frame(t, seed=seed, width=w, height=h, room=room)).cuda() for t in range(n)]


def _snapshot(V, m, X):
    post = m.posterior()
    out = [m.stats(), m.frame_stats(), m.lse(X.shape[0]), post["m"], post["Winv"], post["alpha"]]
    if m.flags_proposal:
        out.append(V.vbgs_proposal_weights(m.ctx))
    return out


@pytest.mark.parametrize("form,flags", [("fp64", 4), ("fp16x3", 4), ("fp16x3", 0), ("fp32", 1)])
def test_save_load_resumes_bit_for_bit(V, tmp_path, form, flags):
    """2k frames uninterrupted against k frames, save, destroy, load, k more
    frames (with the learned proposal: flags 4; plain: 0; caller's order: 1)."""
    K, k = 20_000, 3
    pr = synth.room_prior(K, seed=41)
    frames = _frames(41, 2 * k)
    a = V.Model(pr, form, flags=flags)
    a.flags_proposal = bool(flags & 4)
    ta = [a.update(X, 3) for X in frames]
    ref = _snapshot(V, a, frames[-1])
    a.close()

    b = V.Model(pr, form, flags=flags)
    for X in frames[:k]:
        b.update(X, 3)
    path = str(tmp_path / "state.bin")
    b.save(path)
    S_saved = b.stats()
    b.close()
    c = V.Model.load(path)
    c.flags_proposal = bool(flags & 4)
    assert c.K == K and np.array_equal(c.stats(), S_saved)
    tc = [c.update(X, 3) for X in frames[k:]]
    got = _snapshot(V, c, frames[-1])
    c.close()
    for i in range(k):
        assert np.array_equal(tc[i], ta[k + i]), (i, tc[i], ta[k + i])
    for x, y in zip(got, ref):
        assert np.array_equal(x, y)


def test_save_load_keeps_reassigned_prior(V, tmp_path):
    """The prior means that reassign moved are part of the state."""
    pr = synth.room_prior(3_000, seed=42)
    frames = _frames(42, 3, 64, 64)
    m = V.Model(pr, "fp64")
    m.update(frames[0], 2)
    X = frames[1].cpu().numpy()
    g = np.random.default_rng(3).gumbel(size=X.shape[0])
    _, comps = m.reassign(X, 20, g)
    path = str(tmp_path / "s.bin")
    m.save(path)
    tr_a = m.update(frames[2], 2)
    post_a = m.posterior()
    m.close()
    c = V.Model.load(path)
    tr_c = c.update(frames[2], 2)
    post_c = c.posterior()
    c.close()
    assert np.array_equal(tr_a, tr_c) and np.array_equal(post_a["m"], post_c["m"])
    assert not np.allclose(post_c["m"][comps], O.mstep(pr, np.zeros((3_000, 28)))["m"][comps])


def test_load_refuses_damaged_files(V, tmp_path):
    pr = synth.room_prior(500, seed=43)
    m = V.Model(pr, "fp32")
    m.update(_frames(43, 1, 48, 48)[0], 2)
    path = str(tmp_path / "s.bin")
    m.save(path)
    m.close()
    data = bytearray(open(path, "rb").read())
    assert not os.path.exists(path + ".tmp")
    bad = bytearray(data)
    bad[len(bad) // 2] ^= 0x40
    for blob, name in ((bad, "flip.bin"), (data[:-100], "short.bin"), (b"not a state file at all", "junk.bin")):
        p = tmp_path / name
        p.write_bytes(bytes(blob))
        with pytest.raises(V.VbgsError) as e:
            V.Model.load(str(p))
        assert e.value.code == V.VBGS_EIO
    with pytest.raises(V.VbgsError) as e:
        V.Model.load(str(tmp_path / "missing.bin"))
    assert e.value.code == V.VBGS_EIO
    with pytest.raises(V.VbgsError) as e:
        V.vbgs_save_state(None, str(tmp_path / "x.bin"))
    assert e.value.code == V.VBGS_EINVAL


@pytest.mark.parametrize("form", ["fp64", "fp16x3"])
def test_checks_change_nothing(V, form):
    pr = synth.room_prior(5_000, seed=44)
    frames = _frames(44, 3, 80, 80)
    out = []
    for checks in (False, True):
        m = V.Model(pr, form, checks=checks)
        tr = [m.update(X, 3) for X in frames]
        out.append((np.array(tr), m.stats(), m.launches()))
        m.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[1][2] == out[0][2] + 1       # one check launch per frame


def test_check_kernel_flags_bad_statistics(V):
    X, pr = synth.c1_workload(seed=45, N=3_000, K=200)
    post = O.mstep(pr, np.zeros((200, 28)))
    lse, dS, _ = O.estep_stats(X, post)
    assert V.vbgs_check_frame(dS, X, lse, 1e-9)
    assert V.vbgs_check_frame(dS, np.zeros((0, 6)), None, 1e-9) is False     # counts not conserved
    off = dS.copy()
    off[7, 0] += 0.5                   # a count off by 1.7e-4 of N
    assert not V.vbgs_check_frame(off, X, lse, 1e-6)
    assert V.vbgs_check_frame(off, X, lse, 1e-3)
    for bad in ("nan_stat", "neg", "nan_lse", "moment"):
        d, l = dS.copy(), lse.copy()
        if bad == "nan_stat":
            d[3, 12] = np.nan
        elif bad == "neg":
            d[5, 0] = -1e-3
            d[6, 0] += 1e-3
        elif bad == "nan_lse":
            l[11] = np.inf
        else:
            d[2, 3] += 1e-2 * np.linalg.norm(X.sum(0))
        assert not V.vbgs_check_frame(d, X, l, 1e-6), bad


def test_seed_option(V):
    _, pr = synth.c1_workload(seed=46, N=10, K=2_000)
    w = {}
    for name, seed in (("default", 0), ("a", 7), ("b", 7), ("c", 8)):
        m = V.Model(pr, "fp32", flags=V.VBGS_FLAG_PROPOSAL, seed=seed)
        w[name] = V.vbgs_proposal_weights(m.ctx)
        m.close()
    assert np.array_equal(w["a"], w["b"])
    assert not np.array_equal(w["a"], w["default"]) and not np.array_equal(w["a"], w["c"])
    # He-uniform bound of the first layer: sqrt(6 / 6) = 1
    assert np.max(np.abs(w["a"][:768])) <= 1.0


def test_autotune_cache_option(V, tmp_path):
    """With options.autotune_cache, the first frame of a size class picks the
    work decomposition and appends it to the file; a second context reads it
    back instead of timing, and both give the same results to rounding."""
    pr = synth.room_prior(8_000, seed=47)
    frames = _frames(47, 2, 100, 100)
    import json
    cache = str(tmp_path / "tune.json")
    a = V.Model(pr, "fp16x3", autotune_cache=cache)
    ta = [a.update(X, 2) for X in frames]
    tune_a = V.vbgs_get_tuning(a.ctx)
    Sa = a.stats()
    a.close()
    entries = json.load(open(cache))
    assert len(entries) == 1 and list(entries)[0].startswith("form1_N2^") and tune_a != (0, 0)
    b = V.Model(pr, "fp16x3", autotune_cache=cache)
    tb = [b.update(X, 2) for X in frames]
    assert V.vbgs_get_tuning(b.ctx) == tune_a
    assert O.relerr(np.array(tb), np.array(ta)) <= 1e-12 and O.relerr(b.stats(), Sa) <= 1e-12
    b.close()
    assert json.load(open(cache)) == entries       # read, not re-timed


def test_timeout_leaves_state_unchanged_and_context_usable(V):
    """Failure detection without a fault: with a one-cycle limit, the waits
    between the warp roles of the tensor-core kernels give up as a stalled
    pipeline would; the kernels drain what they issued and return, the frame
    reports VBGS_ETIMEOUT, S_past is unchanged, and with the default limit
    the same context then computes the frame to parity with the oracle."""
    pr = synth.room_prior(2_000, seed=48)
    frames = _frames(48, 2, 64, 64)
    m = V.Model(pr, "fp16x3")
    m.update(frames[0], 2)
    S = m.stats()
    try:
        V.vbgs_set_wait_limit(1)
        with pytest.raises(V.VbgsError) as e:
            m.update(frames[1], 2)
        assert e.value.code == V.VBGS_ETIMEOUT
    finally:
        V.vbgs_set_wait_limit(0)
    assert np.array_equal(m.stats(), S)
    X1 = frames[1].cpu().numpy()
    tr = m.update(frames[1], 2)
    e_ref, S_ref, _, _ = O.cavi_frame(X1, pr, S, 2)
    assert O.relerr(tr, e_ref) <= 1e-4
    for sl in (slice(0, 1), slice(1, 7), slice(7, 28)):
        assert O.relerr(m.stats()[:, sl], S_ref[:, sl]) <= 1e-3
    m.close()
