"""Linear equalities A x = b with free multipliers (the equality block of the
paper's problem class; b'x = 0 of the kernel-learning form) against closed
forms and the FP64 oracle: the KKT linear system of an equality-constrained
QP, the first iterates with a fixed step, full solves of the kernel-learning
form with its bias equality, the smoothed gap, the stand-alone KKT residual
and the coupling pass's equality rows."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2605_29291_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def oracle_params(R, p):
    restart = {R.RESTART_NONE: "none", R.RESTART_FIXED: "fixed", R.RESTART_GAP: "gap"}[p.restart]
    return O.Params(variant="yx" if p.variant == R.YX else "xy", c_nm=p.c_nm, backtracking=bool(p.backtracking),
                    mu=p.mu, c_alpha=p.c_alpha, c_beta=p.c_beta, delta=p.delta, eta=p.eta, tau_bar=p.tau_bar,
                    gamma0=p.gamma0, restart=restart, restart_period=p.restart_period,
                    restart_from_average=bool(p.restart_from_average), xi=p.xi, q=p.q, gap_first=p.gap_first,
                    gap_every=p.gap_every, max_iter=p.max_iter, max_trials=p.max_trials, kkt_every=p.kkt_every,
                    tol=p.tol)


def simplex_params(R, variant=0, **kw):
    return R.Params.default(variant, dual_set=R.DUAL_SIMPLEX, dual_radius=1.0, **kw)


def start(s, data, cuda):
    """x = 0; the simplex centre for the inequality multipliers, 0 for the
    equality multipliers."""
    x = torch.zeros(data.n, dtype=torch.float32, device=cuda)
    y = torch.zeros(s.m, dtype=torch.float32, device=cuda)
    y[:data.m] = 1.0 / data.m
    return x, y


@pytest.fixture(scope="module")
def kml_b():
    return W.kml_minmax(200, 5, 3, seed=1, bias=True)


def test_equality_qp_matches_the_kkt_linear_system(R, cuda):
    """min 0.5 x'Q_0 x + c_0'x s.t. Ax = b (box not active):
    [Q_0 A'; A 0][x; v] = [-c_0; b]."""
    rng = np.random.default_rng(5)
    n, p = 40, 3
    B = rng.standard_normal((n, n))
    Q0 = (B @ B.T / n + 0.3 * np.eye(n)).astype(np.float32)
    Q0 = ((Q0 + Q0.T) * np.float32(0.5)).astype(np.float32)
    c0 = (rng.standard_normal(n) * 0.1).astype(np.float32)
    A = rng.standard_normal((p, n)).astype(np.float32)
    b = (rng.standard_normal(p) * 0.1).astype(np.float32)
    Q64, A64 = Q0.astype(np.float64), A.astype(np.float64)
    K = np.block([[Q64, A64.T], [A64, np.zeros((p, p))]])
    sol = np.linalg.solve(K, np.concatenate([-c0.astype(np.float64), b.astype(np.float64)]))
    xs, vs = sol[:n], sol[n:]
    data = W.QCQPData(n, 0, Q0[None], c0[None], np.zeros(0, np.float32), np.full(n, -50, np.float32),
                      np.full(n, 50, np.float32), A_eq=A, b_eq=b)
    s = R.Solver(data.to(cuda), R.Params.default(R.YX, mu=0.3, tol=1e-8, max_iter=50000, refine=1))
    assert s.m == p
    x = torch.zeros(n, device=cuda)
    y = torch.zeros(p, device=cuda)
    info = s.solve(x, y)
    x64, y64 = s.solution_f64()
    s.close()
    assert info["status"] == R.OK, info
    np.testing.assert_allclose(x64.cpu().numpy(), xs, atol=1e-6 * (1 + np.abs(xs).max()))
    np.testing.assert_allclose(y64.cpu().numpy(), vs, atol=1e-5 * (1 + np.abs(vs).max()))


@pytest.mark.parametrize("variant", [0, 1])
def test_first_iterates_fixed_step(R, cuda, kml_b, variant):
    p = simplex_params(R, variant, backtracking=0, tau_bar=2e-3, tol=0.0, max_iter=50)
    s = R.Solver(kml_b.to(cuda), p)
    s.set_log(50)
    x, y = start(s, kml_b, cuda)
    info = s.solve(x, y, check=False)
    assert info["iters"] == 50
    xl = s.log["x"].cpu().numpy().astype(np.float64)
    yl = s.log["y"].cpu().numpy().astype(np.float64)
    m = s.m
    s.close()
    prob = O.Problem.from_data(kml_b)
    assert prob.m == m
    r = O.rapdb(prob, p=oracle_params(R, p), keep_iterates=50)
    for k, (xo, lo) in enumerate(r.log["iterates"]):
        zo = np.concatenate([xo, lo])
        zg = np.concatenate([xl[k], yl[k, :m]])
        assert np.linalg.norm(zg - zo) <= 1e-5 * max(1.0, np.linalg.norm(zo)), k


@pytest.mark.parametrize("variant,restart", [(0, 1), (0, 2), (1, 1)])
def test_kml_with_bias_matches_oracle(R, cuda, kml_b, variant, restart):
    p = simplex_params(R, variant, restart=restart, restart_period=200, tol=1e-6, max_iter=30000,
                       gap_first=50 if variant == 0 else 100, gap_every=200)
    s = R.Solver(kml_b.to(cuda), p)
    x, y = start(s, kml_b, cuda)
    info = s.solve(x, y)
    x64, y64 = s.solution_f64()
    assert info["status"] == R.OK and info["rel_kkt"] <= 1e-6, info
    prob = O.Problem.from_data(kml_b)
    r = O.rapdb(prob, p=oracle_params(R, p))
    assert r.status == 0
    xg, yg = x64.cpu().numpy(), y64.cpu().numpy()
    fo = prob.phi(r.x, r.lam)
    assert abs(prob.phi(xg, yg) - fo) <= 1e-5 * (1 + abs(fo))
    bvec = kml_b.A_eq[0].astype(np.float64)
    assert abs(bvec @ xg) <= 1e-5 * (1 + np.abs(bvec) @ np.abs(xg))
    rel, _, _ = O.kkt_residual(prob, xg, yg)
    assert rel <= 1.1e-6, rel
    rel_lib, _, _ = s.kkt_residual(x, y)
    ro, _, _ = O.kkt_residual(prob, x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64))
    assert abs(rel_lib - ro) <= 1e-3 * ro + 1e-12
    s.close()


def test_kkt_residual_at_random_points(R, cuda, kml_b):
    s = R.Solver(kml_b.to(cuda), simplex_params(R))
    prob = O.Problem.from_data(kml_b)
    rng = np.random.default_rng(4)
    for k in range(3):
        x = rng.uniform(0, 1, kml_b.n).astype(np.float32)
        y = np.concatenate([rng.dirichlet(np.ones(kml_b.m)), rng.standard_normal(1)]).astype(np.float32)
        rel, rs, rf = s.kkt_residual(torch.from_numpy(x).to(cuda), torch.from_numpy(y).to(cuda))
        ro, rso, rfo = O.kkt_residual(prob, x.astype(np.float64), y.astype(np.float64))
        np.testing.assert_allclose([rel, rs, rf], [ro, rso, rfo], rtol=1e-5)
    s.close()


def test_smoothed_gap_matches_oracle(R, cuda, kml_b):
    p = simplex_params(R, backtracking=0, tau_bar=2e-3, tol=0.0, max_iter=45, restart=R.RESTART_GAP,
                       gap_first=30, gap_every=10)
    s = R.Solver(kml_b.to(cuda), p)
    s.set_log(50)
    x, y = start(s, kml_b, cuda)
    s.solve(x, y, check=False)
    xl = s.log["x"].cpu().numpy().astype(np.float64)
    yl = s.log["y"].cpu().numpy().astype(np.float64)
    G = s.log["gap"].cpu().numpy()
    m = s.m
    s.close()
    prob = O.Problem.from_data(kml_b)
    for e, it in enumerate([30, 40]):
        Go = O.smoothed_gap(prob, xl[it - 1], yl[it - 1, :m], p.xi)
        assert Go > 0
        assert abs(G[e] - Go) <= 2e-3 * abs(Go) + 1e-9, (it, G[e], Go)


def test_coupling_pass_equality_rows(R, cuda, kml_b):
    """The equality rows carry no quadratic term: U and W rows are zero, the
    dots are (0, 0, 0, a'x, a'v)."""
    s = R.Solver(kml_b.to(cuda), simplex_params(R))
    rng = np.random.default_rng(7)
    x = rng.uniform(0, 1, kml_b.n).astype(np.float32)
    v = rng.standard_normal(kml_b.n).astype(np.float32)
    U, Wt, dots = s.coupling_pass(torch.from_numpy(x).to(cuda), torch.from_numpy(v).to(cuda))
    U, Wt, dots = U.cpu().numpy(), Wt.cpu().numpy(), dots.cpu().numpy()
    s.close()
    k = kml_b.m + 1
    assert np.all(U[k] == 0.0) and np.all(Wt[k] == 0.0)
    a = kml_b.A_eq[0].astype(np.float64)
    np.testing.assert_allclose(dots[k, :3], 0.0)
    np.testing.assert_allclose(dots[k, 3], a @ x.astype(np.float64), rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(dots[k, 4], a @ v.astype(np.float64), rtol=1e-12, atol=1e-9)
