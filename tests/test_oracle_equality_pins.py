"""Pins of the oracle's linear equalities (the last rows of the constraint
data, a_k'x - b_k with Q = 0 and a free multiplier): the KKT linear system of
an equality-constrained QP, feasibility and the saddle-value ordering on the
kernel-learning form with the paper's b'x = 0."""
import numpy as np

import oracle as O
from paper_2605_29291_gb300 import workloads as W


def test_equality_qp_matches_the_kkt_linear_system():
    """min 0.5 x'Qx + c'x s.t. Ax = b, box not active: [Q A'; A 0][x; v] = [-c; b]."""
    rng = np.random.default_rng(5)
    n, p = 40, 3
    B = rng.standard_normal((n, n))
    Q = B @ B.T / n + 0.3 * np.eye(n)
    c = rng.standard_normal(n) * 0.1
    A = rng.standard_normal((p, n))
    b = rng.standard_normal(p) * 0.1
    K = np.block([[Q, A.T], [A, np.zeros((p, p))]])
    sol = np.linalg.solve(K, np.concatenate([-c, b]))
    xs, vs = sol[:n], sol[n:]
    assert np.all(np.abs(xs) < 50.0)
    Qs = np.concatenate([Q[None], np.zeros((p, n, n))])
    cs = np.concatenate([c[None], A])
    prob = O.Problem(Qs, cs, -b, -np.full(n, 50.0), np.full(n, 50.0), n_eq=p)
    assert prob.m_ineq == 0
    # (the literal float64 test function cancels below a few 1e-8 here)
    r = O.rapdb(prob, p=O.default_params("yx", mu=0.3, tol=1e-7, max_iter=50000))
    assert r.status == 0, (r.status, r.rel_kkt)
    np.testing.assert_allclose(r.x, xs, atol=1e-5 * (1 + np.abs(xs).max()))
    np.testing.assert_allclose(r.lam, vs, atol=1e-4 * (1 + np.abs(vs).max()))
    assert np.abs(A @ r.x - b).max() <= 1e-6


def test_free_multipliers_are_not_projected():
    prob = O.Problem(np.zeros((3, 2, 2)), np.zeros((3, 2)), np.zeros(2), np.zeros(2), np.ones(2), n_eq=1)
    np.testing.assert_array_equal(prob.proj_y(np.array([-1.0, -2.0])), [0.0, -2.0])
    sx = O.Problem(np.zeros((4, 2, 2)), np.zeros((4, 2)), np.zeros(3), np.zeros(2), np.ones(2),
                   dual_radius=1.0, n_eq=1)
    y = sx.proj_y(np.array([0.5, 0.3, -7.0]))
    np.testing.assert_allclose(y, [0.6, 0.4, -7.0])


def test_kml_minmax_with_the_bias_equality():
    base = W.kml_minmax(120, 5, 3, seed=2)
    eq = W.kml_minmax(120, 5, 3, seed=2, bias=True)
    p0 = O.Problem.from_data(base)
    p1 = O.Problem.from_data(eq)
    assert p1.n_eq == 1 and p1.m == p0.m + 1 and p1.dual_radius == 1.0
    r0 = O.rapdb(p0, p=O.default_params("yx", tol=1e-7, max_iter=50000))
    r1 = O.rapdb(p1, p=O.default_params("yx", tol=1e-7, max_iter=50000))
    assert r0.status == 0 and r1.status == 0
    b = eq.A_eq[0].astype(np.float64)
    assert abs(b @ r1.x) <= 1e-6 * (1 + np.abs(b) @ np.abs(r1.x))
    # min over a smaller set: the saddle value with b'x = 0 is not below the one without
    v0 = p0.f(r0.x) + max(p0.g(r0.x))
    v1 = p1.f(r1.x) + max(p1.g(r1.x)[:p1.m_ineq])
    assert v1 >= v0 - 1e-6 * (1 + abs(v0))
    assert abs(r1.lam[:p1.m_ineq].sum() - 1.0) <= 1e-12
