"""The three-pass mixed-precision search (Sec. 4.2) on CPU: hand-built error
and latency models whose answers follow from the passes' definitions, the
error constraint on random graphs, and a staged numpy computation shaped like
compute_elbo_delta (differences, triangular solve, quadratic form, logit,
log-sum-exp) with each operation's output rounded to its assigned format."""
from __future__ import annotations

import itertools

import numpy as np
import pytest

from paper_2603_08499_gb300 import precision_search as PS

LEVELS = ("fp16", "tf32", "fp32", "fp64")


def additive(errs, times, cast=0.0, edges=()):
    """err(Pi) = sum_i errs[i][Pi_i]; latency = sum_i times[i][Pi_i] + cast per
    edge whose ends sit at different levels."""
    err = lambda c: float(sum(errs[i][c[i]] for i in range(len(c))))
    lat = lambda c: float(sum(times[i][c[i]] for i in range(len(c))) +
                          cast * sum(1 for a, b in edges if c[a] != c[b]))
    return err, lat


def region_model(times, cast, edges):
    """The region and boundary-cast times of the additive model."""
    rt = lambda ops, lv: float(sum(times[i][lv] for i in ops))
    ct = lambda cfg, ops: float(cast * sum(1 for a, b in edges if (a in ops) != (b in ops)))
    return rt, ct


def test_insensitive_operations_all_go_to_the_lowest_precision():
    n = 5
    edges = [(i, i + 1) for i in range(n - 1)]
    err, lat = additive([[0.0] * 4] * n, [[1, 2, 3, 4]] * n, edges=edges)
    p = PS.Problem(n, edges, LEVELS, err, lat, eps=1e-6)
    r = PS.search(p)
    assert r["final"] == (0,) * n and r["map"] == ["fp16"] * n


def test_a_sensitive_operation_is_promoted_to_the_lowest_safe_level():
    eps = 1e-3
    errs = [[1e-5, 1e-6, 0, 0], [5e-2, 4e-3, 2e-4, 0], [1e-5, 1e-6, 0, 0]]   # op 1 is sensitive
    err, lat = additive(errs, [[1, 2, 3, 4]] * 3)
    p = PS.Problem(3, [(0, 1), (1, 2)], LEVELS, err, lat, eps)
    c1 = PS.precision_aware(p)
    # all-low err 5e-2 > eps: op 1 (most sensitive) promoted to fp64; then tried
    # at tf32 (4e-3 + 2e-5 > eps) -> back to fp64; then at fp32 (2e-4 + 2e-5) -> kept
    assert c1 == (0, 2, 0)
    r = PS.search(p)
    assert r["final"] == (0, 2, 0) and r["err"] <= eps


def test_structure_pass_lowers_neighbours_one_level_while_safe():
    eps = 1.0
    errs = [[0.3, 0.2, 0.1, 0], [0.6, 0.5, 0.1, 0], [0.9, 0.1, 0, 0]]
    err, lat = additive(errs, [[1, 2, 3, 4]] * 3)
    p = PS.Problem(3, [(0, 1), (1, 2)], LEVELS, err, lat, eps)
    # seed: op 0 at fp16; op 1 one level down per round while err <= 1:
    # (0,3,3) -> (0,2,3) [0.4] -> (0,1,3)? 0.3+0.5 = 0.8 ok -> (0,0,3)? 0.9 ok; then op 2 from seed 1:
    # (0,0,2)? 0.9 + 0 ok -> (0,0,1)? 1.0 ok -> (0,0,0)? 1.8 no
    c = PS.structure_aware(p, (0, 3, 3))
    assert c == (0, 0, 1) and err(c) <= eps


def test_latency_pass_reverts_regions_whose_casts_cost_more_than_they_save():
    edges = [(0, 1), (1, 2), (2, 3)]
    # op 1 alone at fp16 saves 1 but adds two casts of 2 each: reverted, and
    # at each higher level alone it still costs casts: back to fp64
    times = [[9, 9, 9, 9], [3, 3.5, 4, 4], [9, 9, 9, 9], [9, 9, 9, 9]]
    err, lat = additive([[0, 0, 0, 0]] * 4, times, cast=2.0, edges=edges)
    p = PS.Problem(4, edges, LEVELS, err, lat, 1.0, *region_model(times, 2.0, edges))
    assert PS.latency_aware(p, (3, 0, 3, 3)) == (3, 3, 3, 3)
    # the whole chain at fp16 saves 4 x 1 with no casts inside it: kept
    times2 = [[3, 3.5, 4, 4]] * 4
    err2, lat2 = additive([[0, 0, 0, 0]] * 4, times2, cast=2.0, edges=edges)
    p2 = PS.Problem(4, edges, LEVELS, err2, lat2, 1.0, *region_model(times2, 2.0, edges))
    assert PS.latency_aware(p2, (0, 0, 0, 0)) == (0, 0, 0, 0)
    # without the region callbacks the whole-function comparison charges a cast
    # only where raising removes it: op 1 alone stays where one level up gains nothing
    p3 = PS.Problem(4, edges, LEVELS, err, lat, eps=1.0)
    assert PS.latency_aware(p3, (3, 0, 3, 3)) == (3, 0, 3, 3)


@pytest.mark.parametrize("seed", range(6))
def test_the_final_map_always_meets_the_tolerance(seed):
    rng = np.random.default_rng(seed)
    n = 6
    edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < 0.4]
    errs = [sorted(rng.exponential(1e-3, 4) * [100, 10, 1, 0], reverse=True) for _ in range(n)]
    times = [sorted(rng.uniform(1, 5, 4)) for _ in range(n)]
    cast = float(rng.uniform(0, 1))
    err, lat = additive(errs, times, cast=cast, edges=edges)
    eps = float(rng.uniform(1e-3, 1e-1))
    p = PS.Problem(n, edges, LEVELS, err, lat, eps, *region_model(times, cast, edges))
    r = PS.search(p)
    assert r["err"] <= eps
    # every region kept below fp64 pays for its own casts, so the map is never
    # slower than all-fp64; and it is a feasible point of the brute-force problem
    assert lat(r["final"]) <= lat((3,) * n) + 1e-12
    feasible = [c for c in itertools.product(range(4), repeat=n) if err(c) <= eps]
    assert r["final"] in feasible


def _rounder(level):
    def tf32(a):
        b = np.asarray(a, dtype=np.float32).view(np.uint32)
        return ((b + 0x1000) & 0xFFFFE000).view(np.float32).astype(np.float64)   # 10-bit significand
    return {0: lambda a: np.asarray(a, np.float16).astype(np.float64), 1: tf32,
            2: lambda a: np.asarray(a, np.float32).astype(np.float64), 3: lambda a: np.asarray(a, np.float64)}[level]


def test_search_on_a_staged_logit_and_log_sum_exp():
    """compute_elbo_delta's shape: d = x - m (0), y = L^-1 d (1), q = |y|^2
    (2), l = c - q / 2 (3), lse = log sum exp l (4), each output rounded to
    its format; white-noise inputs, as the paper searches on; latency =
    bytes moved by each operation at its format plus casts."""
    rng = np.random.default_rng(7)
    N, K = 64, 32
    x = rng.standard_normal((N, 6))
    m = rng.standard_normal((K, 6))
    A = rng.standard_normal((K, 6, 6)) * 0.3
    Li = np.tril(A) + 3 * np.eye(6)[None]
    c = rng.standard_normal(K) * 5

    def f(cfg):
        r = [_rounder(lv) for lv in cfg]
        d = r[0](x[:, None, :] - m[None, :, :])
        y = r[1](np.einsum("kij,nkj->nki", Li, d))
        q = r[2](np.sum(y * y, axis=2))
        l = r[3](c[None, :] - 0.5 * q)
        mx = l.max(axis=1, keepdims=True)
        return r[4](mx[:, 0] + np.log(np.exp(l - mx).sum(axis=1)))

    yh = f((3,) * 5)
    err = lambda cfg: float(np.linalg.norm(f(cfg) - yh) / max(np.linalg.norm(yh), 1e-30))
    width = (2, 4, 4, 8)
    sizes = (N * K * 6, N * K * 6, N * K, N * K, N)
    edges = [(0, 1), (1, 2), (2, 3), (3, 4)]
    lat = lambda cfg: float(sum(sizes[i] * width[cfg[i]] for i in range(5)) +
                            sum(sizes[a] for a, b in edges if cfg[a] != cfg[b]))
    rt = lambda ops, lv: float(sum(sizes[i] * width[lv] for i in ops))
    ct = lambda cfg, ops: float(sum(sizes[a] for a, b in edges if (a in ops) != (b in ops)))
    for eps, expect_low in ((1e-6, False), (1e-2, True)):
        p = PS.Problem(5, edges, LEVELS, err, lat, eps, rt, ct)
        r = PS.search(p)
        assert r["err"] <= eps
        assert lat(r["final"]) <= lat((3,) * 5)
        assert (min(r["final"]) == 0) == expect_low, (eps, r["map"])
