"""The kernel-learning problem with the paper's own primal set (Sec. 5.2, eq.
min-max-KML): X = {x >= 0, b'x = 0} with no upper bound, the dual on the
simplex, against the FP64 oracle.  Every trial point and every step of the
smoothed gap's x-subproblem is the projection onto X (the scalar nu of
clamp(v - nu a) on one CTA), and the KKT residual's r_stat is
dist(0, grad + N_X(x)).

* the first iterates with a fixed step, yx and xy;
* full solves (fixed restart, no restart, adaptive restart) by the saddle
  value and the oracle's float64 KKT residual; the iterate stays in X;
* the smoothed gap at logged iterates against the oracle's exact value;
* the stand-alone KKT residual at random points of X;
* packed and quantised storage;
* rejection of a start point off the hyperplane.
"""
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


def kml_params(R, variant=0, **kw):
    base = dict(dual_set=R.DUAL_SIMPLEX, dual_radius=1.0, mu=2.0)
    base.update(kw)
    return R.Params.default(variant, **base)


def start(data, cuda):
    x = torch.zeros(data.n, dtype=torch.float32, device=cuda)
    y = torch.full((data.m,), 1.0 / data.m, dtype=torch.float32, device=cuda)
    return x, y


@pytest.fixture(scope="module")
def kmx():
    return W.kml_minmax(200, 5, 3, seed=1, primal_set=True)


def in_set(data, x):
    a = data.numpy().hyp_a.astype(np.float64)
    return np.all(x >= 0.0) and abs(a @ x) <= 1e-9 * (1.0 + np.abs(a) @ np.abs(x))


@pytest.mark.parametrize("variant", [0, 1])
def test_first_iterates_fixed_step(R, cuda, kmx, variant):
    p = kml_params(R, variant, backtracking=0, tau_bar=2e-3, tol=0.0, max_iter=50, restart=R.RESTART_NONE)
    s = R.Solver(kmx.to(cuda), p)
    s.set_log(50)
    x, y = start(kmx, cuda)
    info = s.solve(x, y, check=False)
    assert info["iters"] == 50
    xl = s.log["x"].cpu().numpy().astype(np.float64)
    yl = s.log["y"].cpu().numpy().astype(np.float64)
    s.close()
    prob = O.Problem.from_data(kmx)
    r = O.rapdb(prob, p=oracle_params(R, p), keep_iterates=50)
    for k, (xo, lo) in enumerate(r.log["iterates"]):
        zo = np.concatenate([xo, lo])
        zg = np.concatenate([xl[k], yl[k, :kmx.m]])
        assert np.linalg.norm(zg - zo) <= 1e-5 * max(1.0, np.linalg.norm(zo)), k


@pytest.mark.parametrize("variant,restart", [(0, 0), (0, 1), (0, 2), (1, 1)])
def test_full_solve_matches_oracle(R, cuda, kmx, variant, restart):
    p = kml_params(R, variant, restart=restart, restart_period=200, tol=1e-6, max_iter=20000,
                   gap_first=50 if variant == 0 else 100, gap_every=200)
    s = R.Solver(kmx.to(cuda), p)
    x, y = start(kmx, cuda)
    info = s.solve(x, y)
    x64, y64 = s.solution_f64()
    assert info["status"] == R.OK and info["rel_kkt"] <= 1e-6, info
    prob = O.Problem.from_data(kmx)
    r = O.rapdb(prob, p=oracle_params(R, p))
    assert r.status == 0
    fo = prob.phi(r.x, r.lam)
    xg, yg = x64.cpu().numpy(), y64.cpu().numpy()
    assert in_set(kmx, xg)
    assert abs(prob.phi(xg, yg) - fo) <= 1e-5 * (1 + abs(fo))
    rel, _, _ = O.kkt_residual(prob, xg, yg)
    assert rel <= 1.1e-6, rel
    s.close()


def test_smoothed_gap_over_the_set(R, cuda, kmx):
    """G_xi at logged iterates (fixed step): the device's accelerated projected
    gradient over X against the oracle's exact x-subproblem."""
    p = kml_params(R, 0, backtracking=0, tau_bar=2e-3, tol=0.0, max_iter=45, restart=R.RESTART_GAP, gap_first=30,
                   gap_every=10)
    s = R.Solver(kmx.to(cuda), p)
    s.set_log(50)
    x, y = start(kmx, cuda)
    info = s.solve(x, y, check=False)
    assert info["iters"] == 45
    xl = s.log["x"].cpu().numpy().astype(np.float64)
    yl = s.log["y"].cpu().numpy().astype(np.float64)
    G = s.log["gap"].cpu().numpy().copy()
    s.close()
    prob = O.Problem.from_data(kmx)
    for e, it in enumerate([30, 40]):
        Go = O.smoothed_gap(prob, xl[it - 1], yl[it - 1, :kmx.m], p.xi)
        assert Go > 0
        assert abs(G[e] - Go) <= 2e-3 * abs(Go) + 1e-9, (it, G[e], Go)


def test_kkt_residual_at_points_of_the_set(R, cuda, kmx):
    prob = O.Problem.from_data(kmx)
    s = R.Solver(kmx.to(cuda), kml_params(R))
    rng = np.random.default_rng(4)
    a = kmx.numpy().hyp_a.astype(np.float64)
    for trial in range(4):
        v = rng.standard_normal(kmx.n) * 0.3
        if trial % 2:
            v = np.abs(v)
        x = O.proj_box_hyperplane(v, prob.lb, prob.ub, a, 0.0)[0].astype(np.float32)
        y = rng.dirichlet(np.ones(kmx.m)).astype(np.float32)
        rel, rs, rf = s.kkt_residual(torch.from_numpy(x).to(cuda), torch.from_numpy(y).to(cuda))
        ro, rso, rfo = O.kkt_residual(prob, x.astype(np.float64), y.astype(np.float64))
        assert abs(rs - rso) <= 1e-5 * (1 + rso), (rs, rso)
        assert abs(rel - ro) <= 1e-5 * (1 + ro), (rel, ro)
    s.close()


@pytest.mark.parametrize("storage,pack", [(0, 1), (1, 1), (2, 0)])
def test_packed_and_quantised_storage(R, cuda, storage, pack):
    data = W.kml_minmax(300, 5, 3, seed=2, primal_set=True)
    p = kml_params(R, 0, restart=R.RESTART_FIXED, restart_period=200, tol=1e-6, max_iter=20000, storage=storage,
                   refine=1, pack_sym=pack)
    s = R.Solver(data.to(cuda), p)
    x, y = start(data, cuda)
    info = s.solve(x, y)
    x64, y64 = s.solution_f64()
    s.close()
    assert info["status"] == R.OK, info
    prob = O.Problem.from_data(data)
    xg, yg = x64.cpu().numpy(), y64.cpu().numpy()
    assert in_set(data, xg)
    rel, _, _ = O.kkt_residual(prob, xg, yg)
    assert rel <= 1.1e-6, rel


def test_start_off_the_hyperplane_rejected(R, cuda, kmx):
    s = R.Solver(kmx.to(cuda), kml_params(R))
    x, y = start(kmx, cuda)
    x[0] = 0.5                     # x >= 0 but b'x = 0.5
    with pytest.raises(R.RapdbError):
        s.solve(x, y)
    s.close()
