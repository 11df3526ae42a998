"""Automatic mixed-precision search (Sec. 4.2): a precision map for the
operations of a staged computation f = f_L o ... o f_1 that minimises the
measured latency T(f^Pi) subject to the relative error of Eq. relerr,
err(Pi) = ||y^h - f^Pi(x)||_2 / max(||y^h||_2, tau) <= eps, against the
all-highest configuration.

The caller describes the computation as operations 0..L-1 with data edges
(producer, consumer), a tuple of candidate precisions ordered lowest first,
and two callbacks on a configuration Pi (one level index per operation):
err(Pi) and latency(Pi) (measured: casts and lost fusion show up in it).  The
search runs the paper's three passes in order:

1. precision-aware: each operation's sensitivity M_p[i] = err(op i alone at
   level p); from the all-lowest configuration, promote operations to the
   highest level in decreasing M_lowest until err <= eps; then, for each
   intermediate level in turn, put the promoted operations at that level and,
   if err > eps, promote them back to the highest in decreasing M_level until
   err <= eps;
2. structure-aware: from the downcast operations as seeds, lower each
   seed's producers and consumers by one level, keeping a change when
   err <= eps; lowered operations become seeds until nothing changes;
3. latency-aware: from the lowest level up, for each cast-bounded region
   C (a connected set of operations at the same reduced level), the net gain
   dT(C) = T_high(C) - (T_low(C) + T_cast(C)): the region's time one level
   higher, at its level, and of the casts at its boundary; with dT <= 0 the
   region moves one level up and is benchmarked again at that level.  The
   region and cast times come from two more callbacks; without them dT is
   taken as T(Pi with C one level up) - T(Pi) on the whole function, which
   charges a cast only where raising the region removes it.

The search itself is host logic: it evaluates the callbacks and never
touches a device.  kernel_problem / search_kernel_map (at the end) build the
callbacks for the library's tensor-core E-step, which run it through the C
ABI.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Sequence

Config = tuple


@dataclass
class Problem:
    n_ops: int
    edges: Sequence[tuple]
    levels: Sequence[str]                  # candidate precisions, lowest first
    err: Callable[[Config], float]
    latency: Callable[[Config], float]
    eps: float
    region_time: Callable[[Sequence[int], int], float] | None = None   # T of ops at a level
    cast_time: Callable[[Config, Sequence[int]], float] | None = None  # casts at a region's boundary
    evaluations: int = field(default=0, init=False)

    def e(self, cfg: Config) -> float:
        self.evaluations += 1
        return self.err(tuple(cfg))

    @property
    def top(self) -> int:
        return len(self.levels) - 1

    def neighbours(self, i: int) -> list:
        return sorted({b for a, b in self.edges if a == i} | {a for a, b in self.edges if b == i})


def _set(cfg, ops, level) -> Config:
    c = list(cfg)
    for i in ops:
        c[i] = level
    return tuple(c)


def sensitivities(p: Problem) -> dict:
    """M[level][i] = err(op i alone at level, all others highest)."""
    high = tuple([p.top] * p.n_ops)
    return {lv: [p.e(_set(high, [i], lv)) for i in range(p.n_ops)] for lv in range(p.top)}


def precision_aware(p: Problem, M: dict | None = None) -> Config:
    M = sensitivities(p) if M is None else M
    cfg = tuple([0] * p.n_ops)
    promoted = []

    def promote(cfg, candidates, scores):
        order = sorted(candidates, key=lambda i: (-scores[i], i))   # most sensitive first, ties by index
        for i in order:
            if p.e(cfg) <= p.eps:
                break
            cfg = _set(cfg, [i], p.top)
        return cfg

    if p.e(cfg) > p.eps:
        before = cfg
        cfg = promote(cfg, range(p.n_ops), M[0])
        promoted = [i for i in range(p.n_ops) if before[i] != cfg[i]]
    for lv in range(1, p.top):
        if not promoted:
            break
        trial = _set(cfg, promoted, lv)
        if p.e(trial) <= p.eps:
            cfg = trial
            promoted = []      # every promoted operation now sits at this level
            break
        cfg = promote(trial, promoted, M[lv])
        promoted = [i for i in promoted if cfg[i] == p.top]
    return cfg


def structure_aware(p: Problem, cfg: Config) -> Config:
    seeds = [i for i in range(p.n_ops) if cfg[i] < p.top]
    while seeds:
        new = []
        for s in seeds:
            for j in p.neighbours(s):
                if cfg[j] == 0:
                    continue
                trial = _set(cfg, [j], cfg[j] - 1)
                if p.e(trial) <= p.eps:
                    cfg = trial
                    new.append(j)
        seeds = sorted(set(new))
    return cfg


def regions(p: Problem, cfg: Config, level: int) -> list:
    """Connected sets of operations at `level` (edges within the set)."""
    todo = {i for i in range(p.n_ops) if cfg[i] == level}
    out = []
    while todo:
        stack, comp = [min(todo)], set()
        while stack:
            i = stack.pop()
            if i in comp:
                continue
            comp.add(i)
            stack.extend(j for j in p.neighbours(i) if j in todo and j not in comp)
        todo -= comp
        out.append(sorted(comp))
    return out


def latency_aware(p: Problem, cfg: Config) -> Config:
    for lv in range(p.top):
        for reg in regions(p, cfg, lv):
            raised = _set(cfg, reg, lv + 1)
            if p.region_time is not None and p.cast_time is not None:
                gain = p.region_time(reg, lv + 1) - (p.region_time(reg, lv) + p.cast_time(cfg, reg))
            else:
                gain = p.latency(raised) - p.latency(cfg)
            if gain <= 0.0:
                cfg = raised
    return cfg


def search(p: Problem) -> dict:
    """Pi* and the configuration after each pass."""
    c1 = precision_aware(p)
    c2 = structure_aware(p, c1)
    c3 = latency_aware(p, c2)
    return {"precision_aware": c1, "structure_aware": c2, "final": c3,
            "map": [p.levels[i] for i in c3], "err": p.err(c3), "evaluations": p.evaluations}


# ---------------------------------------------------------------------------
# The search applied to the library's tensor-core E-step: its operations are
# the six lo terms of the hi/lo products (vbgs.KNOBS: pass-1 features and
# coefficients, pass-2 recomputed-logit features and coefficients, pass-2
# responsibilities and statistics features), each at level "hi" (the term
# left out) or "hi+lo" (kept).  err is Eq. relerr of the E-step's outputs --
# the per-point lse_n and the statistics N, S1, S2 of one iteration -- against
# the FP64 form from the same state; latency the measured device time of the
# two passes.  Edges: the operands of one product, and the operands the two
# passes share (the point features, the coefficient tiles, the logits that
# make the responsibilities).
# ---------------------------------------------------------------------------
KNOB_EDGES = [(0, 1), (2, 3), (4, 5), (0, 2), (1, 3), (3, 4)]


def knobs_of(cfg) -> int:
    """Knob bits of a configuration: bit i set where op i is at level 0 (hi)."""
    return sum(1 << i for i, lv in enumerate(cfg) if lv == 0)


def kernel_problem(V, prior, S, X, eps: float, form: str = "fp16x3", reps: int = 3) -> Problem:
    """A Problem over the tensor-core E-step's knobs on the frame X (device
    N x 6) from the statistics S.  The callbacks run the library."""
    import numpy as np

    def run(form_, knobs, profile):
        m = V.Model(prior, form_)
        if knobs:
            V.vbgs_set_precision_knobs(m.ctx, knobs)
        m.set_stats(S)
        if profile:
            m.profile(V.prof_only(0, 2))
            m.profile_read(reset=True)
        tr = m.update(X, 1)
        out = (tr, m.lse(X.shape[0]), m.frame_stats())
        ms = None
        if profile:
            p = m.profile_read()
            ms = p["pass1"][0] + p["pass2"][0]
        m.close()
        return out, ms

    ref, _ = run("fp64", 0, False)

    def rel(a, b):
        a, b = np.asarray(a, dtype=np.float64).ravel(), np.asarray(b, dtype=np.float64).ravel()
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))

    cache = {}

    def err(cfg):
        k = knobs_of(cfg)
        if k not in cache:
            try:
                (tr, lse, dS), _ = run(form, k, False)
                e = max(rel(lse, ref[1]), rel(dS[:, 0], ref[2][:, 0]), rel(dS[:, 1:7], ref[2][:, 1:7]),
                        rel(dS[:, 7:], ref[2][:, 7:]), rel(tr, ref[0]))
                cache[k] = e if np.isfinite(e) else float("inf")
            except V.VbgsError:
                # statistics so far off that a posterior is not positive
                # definite (or non-finite): no tolerance admits the map
                cache[k] = float("inf")
        return cache[k]

    def latency(cfg):
        k = knobs_of(cfg)
        try:
            return float(np.median([run(form, k, True)[1] for _ in range(reps)]))
        except V.VbgsError:
            return float("inf")

    return Problem(n_ops=6, edges=KNOB_EDGES, levels=("hi", "hi+lo"), err=err, latency=latency, eps=eps)


def search_kernel_map(V, prior, S, X, eps: float = 1e-6, form: str = "fp16x3") -> dict:
    """Run the three passes on the library's knobs; the result's "knobs" is
    the map for vbgs_set_precision_knobs, with its error and the latency of
    the all-kept and the chosen maps."""
    p = kernel_problem(V, prior, S, X, eps, form)
    res = search(p)
    full = tuple([1] * 6)
    res["knobs"] = knobs_of(res["final"])
    res["left_out"] = [V.KNOBS[i] for i in range(6) if res["final"][i] == 0]
    res["err_all_kept"] = p.err(full)
    res["eps"] = eps
    res["feasible"] = res["err"] <= eps
    res["latency_ms"] = p.latency(res["final"])
    res["latency_ms_all_kept"] = p.latency(full)
    for k in ("precision_aware", "structure_aware", "final"):
        res[k] = list(res[k])
    return res
