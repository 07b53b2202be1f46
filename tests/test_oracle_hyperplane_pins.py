"""Pins of the oracle's primal set with one hyperplane, X = {lb <= x <= ub,
a'x = beta} (the kernel-learning problem of Sec. 5.2, eq. min-max-KML,
minimises over {x >= 0, b'x = 0}), against computations that do not go
through the oracle:

* the projection onto X against exhaustive active-set enumeration (every
  free / lower / upper pattern, the equality solved on the free set) and
  against its optimality conditions;
* the distance dist(0, g + N_X(x)) in the KKT residual against a golden-section
  minimisation of the same convex function of t, and against the closed form
  when no coordinate is at a bound;
* the smoothed gap's x-subproblem over X against exhaustive enumeration of
  the equality-constrained QP on every active pattern;
* a whole rAPDB run with one constraint (the simplex dual is then {1}, so the
  min-max problem is the QP min_{x in X} f + g_1) against that QP solved by
  enumeration.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from paper_2605_29291_gb300 import workloads as W


def brute_projection(v, lb, ub, a, beta):
    """argmin ||x - v|| over {lb <= x <= ub, a'x = beta} by enumeration."""
    n = v.size
    best, bx = math.inf, None
    for pat in itertools.product((0, 1, 2), repeat=n):
        if any(p == 2 and not np.isfinite(ub[j]) for j, p in enumerate(pat)):
            continue
        if any(p == 1 and not np.isfinite(lb[j]) for j, p in enumerate(pat)):
            continue
        x = v.copy()
        F = np.array([p == 0 for p in pat])
        for j, p in enumerate(pat):
            if p == 1:
                x[j] = lb[j]
            elif p == 2:
                x[j] = ub[j]
        aF = a[F]
        rest = beta - a[~F] @ x[~F]
        den = aF @ aF
        if den > 0:
            nu = (aF @ v[F] - rest) / den
            x[F] = v[F] - nu * aF
        elif abs(rest - aF @ v[F]) > 1e-12:
            continue
        if np.all(x >= lb - 1e-12) and np.all(x <= ub + 1e-12) and abs(a @ x - beta) <= 1e-9:
            d = float(np.sum((x - v) ** 2))
            if d < best:
                best, bx = d, x
    return bx


def random_case(rng, n, inf_ub):
    lb = rng.uniform(-2, 0, n)
    ub = np.full(n, np.inf) if inf_ub else lb + rng.uniform(0.5, 3, n)
    a = rng.standard_normal(n)
    a[rng.random(n) < 0.2] = 0.0
    if not np.any(a):
        a[0] = 1.0
    x_feas = lb + rng.uniform(0, 1, n) * (np.minimum(ub, lb + 3) - lb)
    beta = float(a @ x_feas)                     # a point of the box on the hyperplane
    v = rng.standard_normal(n) * 3
    return v, lb, ub, a, beta


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("inf_ub", [False, True])
def test_projection_matches_enumeration(seed, inf_ub):
    rng = np.random.default_rng(seed)
    n = 2 + seed % 5
    v, lb, ub, a, beta = random_case(rng, n, inf_ub)
    x, nu = O.proj_box_hyperplane(v, lb, ub, a, beta)
    xb = brute_projection(v, lb, ub, a, beta)
    np.testing.assert_allclose(x, xb, rtol=1e-10, atol=1e-10)
    # optimality: v - x = nu a + mu with mu in N_box(x) (<= 0 at lb, >= 0 at ub, 0 inside)
    mu = v - x - nu * a
    inside = (x > lb) & (x < ub)
    assert np.all(np.abs(mu[inside]) <= 1e-9)
    assert np.all(mu[(x <= lb) & ~inside] <= 1e-9) and np.all(mu[(x >= ub) & ~inside] >= -1e-9)
    assert abs(a @ x - beta) <= 1e-9 * (1 + np.abs(a) @ np.abs(x))


def test_projection_of_the_kernel_learning_set():
    """{x >= 0, b'x = 0} with b = +-1 labels: projecting a point of the set
    returns it; the projection of v has equal class sums."""
    rng = np.random.default_rng(3)
    n = 40
    b = np.ones(n)
    b[n // 2:] = -1
    lb, ub = np.zeros(n), np.full(n, np.inf)
    v = rng.standard_normal(n)
    x, _ = O.proj_box_hyperplane(v, lb, ub, b, 0.0)
    assert np.all(x >= 0) and abs(x[:n // 2].sum() - x[n // 2:].sum()) <= 1e-12
    x2, _ = O.proj_box_hyperplane(x, lb, ub, b, 0.0)
    np.testing.assert_allclose(x2, x, atol=1e-14)


def golden_min(F, lo, hi, iters=300):
    g = (math.sqrt(5) - 1) / 2
    a_, b_ = lo, hi
    c_, d_ = b_ - g * (b_ - a_), a_ + g * (b_ - a_)
    for _ in range(iters):
        if F(c_) < F(d_):
            b_ = d_
        else:
            a_ = c_
        c_, d_ = b_ - g * (b_ - a_), a_ + g * (b_ - a_)
    t = 0.5 * (a_ + b_)
    return F(t), t


@pytest.mark.parametrize("seed", range(10))
def test_cone_distance_matches_golden_section(seed):
    rng = np.random.default_rng(100 + seed)
    n = 8
    lb, ub = np.zeros(n), np.where(rng.random(n) < 0.5, np.inf, 2.0)
    x = np.where(rng.random(n) < 0.4, 0.0, rng.uniform(0.1, 1.9, n))
    x = np.where((rng.random(n) < 0.2) & np.isfinite(ub), ub, x)
    g = rng.standard_normal(n)
    a = rng.standard_normal(n)

    def F(t):
        r = np.where(x <= lb, np.maximum(-(g + t * a), 0.0),
                     np.where(x >= ub, np.maximum(g + t * a, 0.0), np.abs(g + t * a)))
        return float(np.sum(r * r))
    ref, _ = golden_min(F, -1e3, 1e3)
    d, t = O.hyperplane_cone_distance(g, x, lb, ub, a)
    assert abs(d * d - ref) <= 1e-9 * (1 + ref)
    assert abs(F(t) - d * d) <= 1e-12 * (1 + ref)


def test_cone_distance_interior_closed_form():
    rng = np.random.default_rng(7)
    n = 10
    lb, ub = np.zeros(n), np.full(n, np.inf)
    x = rng.uniform(0.5, 1.0, n)
    g, a = rng.standard_normal(n), rng.standard_normal(n)
    d, t = O.hyperplane_cone_distance(g, x, lb, ub, a)
    proj = g - (a @ g) / (a @ a) * a
    assert abs(d - np.linalg.norm(proj)) <= 1e-12 and abs(t + (a @ g) / (a @ a)) <= 1e-12


def brute_eq_qp(H, lin, lb, ub, a, beta):
    """min 0.5 x'Hx + lin'x over {lb <= x <= ub, a'x = beta}, H positive
    definite, by enumerating active patterns and solving the KKT system
    [H_FF a_F; a_F' 0] on the free set."""
    n = lin.size
    best, bx = math.inf, None
    for pat in itertools.product((0, 1, 2), repeat=n):
        if any(p == 2 and not np.isfinite(ub[j]) for j, p in enumerate(pat)):
            continue
        x = np.zeros(n)
        F = np.array([p == 0 for p in pat])
        for j, p in enumerate(pat):
            if p == 1:
                x[j] = lb[j]
            elif p == 2:
                x[j] = ub[j]
        k = int(F.sum())
        fx = ~F
        rhs_eq = beta - a[fx] @ x[fx]
        if k == 0:
            if abs(rhs_eq) > 1e-10:
                continue
        else:
            K = np.zeros((k + 1, k + 1))
            K[:k, :k] = H[np.ix_(F, F)]
            K[:k, k] = a[F]
            K[k, :k] = a[F]
            r = np.concatenate([-(lin[F] + H[np.ix_(F, fx)] @ x[fx]), [rhs_eq]])
            try:
                sol = np.linalg.solve(K, r)
            except np.linalg.LinAlgError:
                continue
            x[F] = sol[:k]
        if np.all(x >= lb - 1e-10) and np.all(x <= ub + 1e-10) and abs(a @ x - beta) <= 1e-8:
            val = 0.5 * x @ H @ x + lin @ x
            if val < best:
                best, bx = val, x
    return bx


@pytest.mark.parametrize("seed", range(4))
def test_gap_subproblem_over_the_set_matches_enumeration(seed):
    rng = np.random.default_rng(seed)
    n = 5
    d = W.kml_minmax(n, 3, 3, seed=seed, primal_set=True)
    prob = O.Problem.from_data(d)
    x = np.abs(rng.standard_normal(n))
    x = O.proj_box_hyperplane(x, prob.lb, prob.ub, prob.hyp[0], prob.hyp[1])[0]
    lam = rng.dirichlet(np.ones(prob.m))
    xi = 0.04
    H = prob.Q[0] + np.tensordot(lam, prob.Q[1:], axes=1) + 2 * xi * np.eye(n)
    lin = prob.c[0] + lam @ prob.c[1:] - 2 * xi * x
    xb = brute_eq_qp(H, lin, prob.lb, prob.ub, prob.hyp[0], prob.hyp[1])
    xs = O.gap_x_subproblem(prob, x, lam, xi)
    np.testing.assert_allclose(xs, xb, rtol=1e-7, atol=1e-9)


def test_rapdb_over_the_set_matches_the_qp_with_one_constraint():
    """m = 1: the dual simplex is {1}, and min-max-KML is the QP
    min_{x >= 0, b'x = 0} lam |x|^2 - 2 1'x + m x'H x."""
    n = 6
    rng = np.random.default_rng(11)
    A = rng.standard_normal((n, n))
    H1 = A @ A.T / n
    b = np.array([1, 1, 1, -1, -1, -1], np.float64)
    Q = np.zeros((2, n, n))
    Q[0] = 2.0 * np.eye(n)
    Q[1] = 2.0 * H1
    c = np.zeros((2, n))
    c[0] = -2.0
    prob = O.Problem(Q, c, np.zeros(1), np.zeros(n), np.full(n, np.inf), dual_radius=1.0,
                     hyperplane=(b, 0.0))
    p = O.default_params("yx", mu=2.0, restart="none", tol=1e-6, max_iter=20000)
    r = O.rapdb(prob, lam0=np.ones(1), p=p)
    assert r.status == 0
    xb = brute_eq_qp(Q[0] + Q[1], c[0] + c[1], prob.lb, prob.ub, b, 0.0)
    np.testing.assert_allclose(r.x, xb, atol=1e-5)
    assert np.all(r.x >= 0) and abs(b @ r.x) <= 1e-12
