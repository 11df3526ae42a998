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

Host logic only: it evaluates the callbacks and never touches a device.
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
