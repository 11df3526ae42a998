"""GPU tests of the per-operation precision knobs of the tensor-core E-step
and of the mixed-precision search (Sec. 4.2) run on them.

Each knob leaves one lo term out of the hi/lo products; with every term kept
(knobs 0) the form is the default one, bit for bit.  Leaving a term out can
only lose accuracy against the FP64 form, never gain it beyond rounding.  The
search returns a map whose measured error (Eq. relerr of lse and the
statistics of one iteration, against the FP64 form from the same state)
meets the tolerance when any map does, and keeps every term when none does.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2603_08499_gb300 import synth
from paper_2603_08499_gb300 import precision_search as PS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    from paper_2603_08499_gb300 import build
    build.build()
    from paper_2603_08499_gb300 import vbgs
    return vbgs


@pytest.fixture(scope="module")
def setup(V):
    import torch
    room = synth.Room(61)
    pr = synth.room_prior(3_000, seed=61)
    m = V.Model(pr, "fp64")
    for t in range(2):
        m.update(synth.room_frame(t, seed=61, width=80, height=80, room=room), 2)
    S = m.stats()
    m.close()
    X = torch.from_numpy(synth.room_frame(2, seed=61, width=80, height=80, room=room)).cuda()
    return pr, S, X


def test_knobs_zero_is_the_default_form(V, setup):
    pr, S, X = setup
    out = []
    for knobs in (None, 0):
        m = V.Model(pr, "fp16x3")
        if knobs is not None:
            V.vbgs_set_precision_knobs(m.ctx, knobs)
        m.set_stats(S)
        out.append((m.update(X, 2), m.stats()))
        m.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    with pytest.raises(V.VbgsError):
        m = V.Model(pr, "fp16x3")
        try:
            V.vbgs_set_precision_knobs(m.ctx, 64)
        finally:
            m.close()


def test_each_knob_loses_accuracy(V, setup):
    pr, S, X = setup
    p = PS.kernel_problem(V, pr, S, X, eps=1e-6)
    full = p.err((1,) * 6)
    assert full < 1e-4
    for i in range(6):
        cfg = [1] * 6
        cfg[i] = 0
        e = p.err(tuple(cfg))
        assert e >= 0.5 * full, (V.KNOBS[i], e, full)
    # every lo term out: hi-only FP16 operands on expanded quadratic forms
    assert p.err((0,) * 6) > 100 * full


@pytest.mark.parametrize("eps", [1e-6, 1e-3])
def test_search_returns_a_map_within_tolerance(V, setup, eps):
    pr, S, X = setup
    res = PS.search_kernel_map(V, pr, S, X, eps=eps)
    if res["feasible"]:
        assert res["err"] <= eps
    else:
        assert res["knobs"] == 0 and res["err_all_kept"] > eps
    # the chosen map, set on a context, reproduces the measured error
    p = PS.kernel_problem(V, pr, S, X, eps)
    assert abs(p.err(tuple(res["final"])) - res["err"]) <= 1e-12 + 1e-9 * res["err"]
    assert res["latency_ms"] > 0 and res["evaluations"] > 6
