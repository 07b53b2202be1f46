"""Pins of the oracle's simplex-dual parts (the kernel-learning min-max problem
of Sec. 5.2 with y in {y >= 0, sum y = r}) against facts fixed by the
mathematics, not by the oracle itself: an independent bisection for the
projection, a grid minimisation for the normal-cone distance, the m = 1 closed
form, brute force on a tiny minimax, and the optimality conditions."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2605_29291_gb300 import workloads as W


def proj_bisect(v, r):
    """The projection is max(v - theta, 0) with sum = r; the sum is
    continuous and decreasing in theta, so bisection finds theta."""
    lo, hi = v.min() - r, v.max()
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.maximum(v - mid, 0.0).sum() > r:
            lo = mid
        else:
            hi = mid
    return np.maximum(v - 0.5 * (lo + hi), 0.0)


@pytest.mark.parametrize("seed", range(5))
def test_simplex_projection_against_bisection(seed):
    rng = np.random.default_rng(seed)
    for m in (1, 2, 3, 7, 20):
        v = rng.standard_normal(m) * 3.0
        r = float(rng.uniform(0.5, 2.0))
        y = O.proj_simplex(v, r)
        np.testing.assert_allclose(y, proj_bisect(v, r), atol=1e-12)
        assert np.all(y >= 0.0) and abs(y.sum() - r) <= 1e-12 * max(1.0, r)
        np.testing.assert_allclose(O.proj_simplex(y, r), y, atol=1e-14)       # idempotent


def test_simplex_projection_worked_example():
    # v = (0.5, 0.3, -0.2), r = 1: theta = (0.5 + 0.3 - 1) / 2 = -0.1
    np.testing.assert_allclose(O.proj_simplex(np.array([0.5, 0.3, -0.2]), 1.0), [0.6, 0.4, 0.0], atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_simplex_cone_distance_against_grid(seed):
    rng = np.random.default_rng(seed + 10)
    for m in (1, 2, 4, 9):
        g = rng.standard_normal(m)
        lam = np.where(rng.uniform(size=m) < 0.5, rng.uniform(0.1, 1.0, m), 0.0)
        if not lam.any():
            lam[0] = 1.0
        d, t = O.simplex_cone_distance(g, lam)
        on = lam > 0

        def F(tt):
            return float(np.sum((g[on] - tt) ** 2) + np.sum(np.maximum(g[~on] - tt, 0.0) ** 2))
        ts = np.linspace(g.min() - 1.0, g.max() + 1.0, 200001)
        grid = min(F(tt) for tt in ts[::50])
        # fine grid around the coarse minimiser
        tc = ts[::50][int(np.argmin([F(tt) for tt in ts[::50]]))]
        fine = min(F(tt) for tt in np.linspace(tc - 1e-3, tc + 1e-3, 2001))
        assert d * d <= min(grid, fine) + 1e-12
        assert abs(d * d - fine) <= 1e-6
        assert abs(F(t) - d * d) <= 1e-12


def test_simplex_cone_distance_zero_exactly_at_optimal_duals():
    g = np.array([1.0, 1.0, 0.5, -2.0])
    assert O.simplex_cone_distance(g, np.array([0.3, 0.7, 0.0, 0.0]))[0] == 0.0
    # mass on a non-maximal constraint is not optimal
    assert O.simplex_cone_distance(g, np.array([0.5, 0.0, 0.5, 0.0]))[0] > 0.1


def test_single_constraint_reduces_to_a_box_qp_closed_form():
    """With m = 1 the simplex is {1}: the problem is min f + g_1 over the box;
    for an interior solution x* = -(Q_0 + Q_1)^{-1}(c_0 + c_1)."""
    rng = np.random.default_rng(3)
    n = 30
    A0, A1 = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    Q0 = A0 @ A0.T / n + 0.5 * np.eye(n)
    Q1 = A1 @ A1.T / n
    c = rng.standard_normal((2, n)) * 0.1
    prob = O.Problem(np.stack([Q0, Q1]), c, np.array([0.0]), -np.full(n, 50.0), np.full(n, 50.0), dual_radius=1.0)
    xs = -np.linalg.solve(Q0 + Q1, c[0] + c[1])
    assert np.all(np.abs(xs) < 50.0)
    # (tolerances near 1e-9 are out of reach of the literal float64 test
    # function: its Phi differences cancel)
    r = O.rapdb(prob, p=O.default_params("yx", mu=0.5, tol=1e-8, max_iter=20000))
    assert r.status == 0
    np.testing.assert_allclose(r.x, xs, atol=1e-7 * (1 + np.abs(xs).max()))
    np.testing.assert_allclose(r.lam, [1.0])


def test_tiny_minimax_against_brute_force():
    """n = 2, m = 2 on [0, 1]^2: min_x f(x) + max(g_1(x), g_2(x)) (the max over
    the 2-simplex of y'g) by a grid, against the oracle's saddle point."""
    Q0 = np.array([[2.0, 0.0], [0.0, 2.0]])
    Q1 = np.array([[4.0, 1.0], [1.0, 1.0]])
    Q2 = np.array([[1.0, -0.5], [-0.5, 3.0]])
    c = np.array([[-2.0, -2.0], [0.0, 0.0], [0.0, 0.0]])
    prob = O.Problem(np.stack([Q0, Q1, Q2]), c, np.zeros(2), np.zeros(2), np.ones(2), dual_radius=1.0)
    r = O.rapdb(prob, p=O.default_params("yx", mu=2.0, tol=1e-7, max_iter=50000))
    assert r.status == 0

    def val(x):
        return prob.f(x) + max(prob.g(x))
    ts = np.linspace(0.0, 1.0, 1001)
    X, Y = np.meshgrid(ts, ts, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel()], 1)
    vals = np.array([val(p) for p in pts])
    best = vals.min()
    assert abs(val(r.x) - best) <= 1e-5
    # the dual weights sit on the active constraints
    g = prob.g(r.x)
    assert abs(r.lam.sum() - 1.0) <= 1e-12 and np.all(r.lam >= 0)
    assert np.all(g[r.lam > 1e-6] >= g.max() - 1e-6)


def test_kml_minmax_converges_and_the_gap_vanishes():
    data = W.kml_minmax(120, 5, 3, seed=2)
    prob = O.Problem.from_data(data)
    assert prob.dual_radius == 1.0
    r = O.rapdb(prob, p=O.default_params("yx", tol=1e-7, max_iter=20000))
    assert r.status == 0 and r.rel_kkt <= 1e-7
    assert abs(r.lam.sum() - 1.0) <= 1e-12 and np.all(r.lam >= 0.0)
    G = O.smoothed_gap(prob, r.x, r.lam, 0.04)
    assert -1e-9 <= G <= 1e-5
    rng = np.random.default_rng(0)
    x = np.clip(r.x + 0.05 * rng.standard_normal(prob.n), prob.lb, prob.ub)
    lam = O.proj_simplex(r.lam + 0.2 * rng.standard_normal(prob.m), 1.0)
    assert O.smoothed_gap(prob, x, lam, 0.04) > 0.0
    assert math.isfinite(O.kkt_residual(prob, x, lam)[0])
