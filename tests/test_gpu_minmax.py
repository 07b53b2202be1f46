"""The dual on a simplex (the kernel-learning min-max problem of Sec. 5.2)
against the FP64 oracle: the first iterates with a fixed step, full solves
(objective and the oracle's float64 KKT residual), the smoothed gap, the
stand-alone KKT residual, the xy variant, input validation, and the full-size
n = 5000, m = 8 instance in BF16 with refinement."""
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


def start(data, cuda):
    x = torch.zeros(data.n, dtype=torch.float32, device=cuda)
    y = torch.full((data.m,), 1.0 / data.m, dtype=torch.float32, device=cuda)
    return x, y


@pytest.fixture(scope="module")
def kml():
    return W.kml_minmax(200, 5, 3, seed=1)


@pytest.mark.parametrize("variant", [0, 1])
def test_first_iterates_fixed_step(R, cuda, kml, variant):
    p = simplex_params(R, variant, backtracking=0, tau_bar=2e-3, tol=0.0, max_iter=50)
    s = R.Solver(kml.to(cuda), p)
    s.set_log(50)
    x, y = start(kml, cuda)
    info = s.solve(x, y, check=False)
    assert info["iters"] == 50
    xl = s.log["x"].cpu().numpy().astype(np.float64)
    yl = s.log["y"].cpu().numpy().astype(np.float64)
    s.close()
    prob = O.Problem.from_data(kml)
    r = O.rapdb(prob, p=oracle_params(R, p), keep_iterates=50)
    for k, (xo, lo) in enumerate(r.log["iterates"]):
        zo = np.concatenate([xo, lo])
        zg = np.concatenate([xl[k], yl[k, :kml.m]])
        assert np.linalg.norm(zg - zo) <= 1e-5 * max(1.0, np.linalg.norm(zo)), k
        assert abs(yl[k, :kml.m].sum() - 1.0) <= 1e-6 and np.all(yl[k] >= 0.0)


@pytest.mark.parametrize("variant,restart", [(0, 1), (0, 2), (1, 1)])
def test_full_solve_matches_oracle(R, cuda, kml, variant, restart):
    p = simplex_params(R, variant, restart=restart, restart_period=200, tol=1e-6, max_iter=20000,
                       gap_first=50 if variant == 0 else 100, gap_every=200)
    s = R.Solver(kml.to(cuda), p)
    x, y = start(kml, cuda)
    info = s.solve(x, y)
    x64, y64 = s.solution_f64()
    assert info["status"] == R.OK and info["rel_kkt"] <= 1e-6, info
    prob = O.Problem.from_data(kml)
    r = O.rapdb(prob, p=oracle_params(R, p))
    assert r.status == 0
    fo = prob.f(r.x) + float(r.lam @ prob.g(r.x))                 # the saddle value
    xg, yg = x64.cpu().numpy(), y64.cpu().numpy()
    assert abs(prob.phi(xg, yg) - fo) <= 1e-5 * (1 + abs(fo))
    assert abs(yg.sum() - 1.0) <= 1e-12 and np.all(yg >= 0.0)
    rel, _, _ = O.kkt_residual(prob, xg, yg)
    assert rel <= 1.1e-6, rel
    # the stand-alone residual at the returned float32 point matches the oracle's
    rel_lib, rs_lib, rf_lib = s.kkt_residual(x, y)
    ro, rso, rfo = O.kkt_residual(prob, x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64))
    assert abs(rel_lib - ro) <= 1e-3 * ro + 1e-12
    s.close()


def test_kkt_residual_at_random_points(R, cuda, kml):
    s = R.Solver(kml.to(cuda), simplex_params(R))
    prob = O.Problem.from_data(kml)
    rng = np.random.default_rng(4)
    for k in range(4):
        x = rng.uniform(0, 1, kml.n).astype(np.float32)
        x[:5] = 0.0
        x[5:9] = 1.0
        y = rng.uniform(0, 1, kml.m)
        if k % 2:
            y[0] = 0.0
        y = (y / y.sum()).astype(np.float32)
        rel, rs, rf = s.kkt_residual(torch.from_numpy(x).to(cuda), torch.from_numpy(y).to(cuda))
        ro, rso, rfo = O.kkt_residual(prob, x.astype(np.float64), y.astype(np.float64))
        np.testing.assert_allclose([rel, rs, rf], [ro, rso, rfo], rtol=1e-5)
    s.close()


def test_smoothed_gap_matches_oracle(R, cuda, kml):
    p = simplex_params(R, backtracking=0, tau_bar=2e-3, tol=0.0, max_iter=45, restart=R.RESTART_GAP,
                       gap_first=30, gap_every=10)
    s = R.Solver(kml.to(cuda), p)
    s.set_log(50)
    x, y = start(kml, cuda)
    info = s.solve(x, y, check=False)
    assert info["iters"] == 45
    xl = s.log["x"].cpu().numpy().astype(np.float64)
    yl = s.log["y"].cpu().numpy().astype(np.float64)
    G = s.log["gap"].cpu().numpy()
    s.close()
    prob = O.Problem.from_data(kml)
    for e, it in enumerate([30, 40]):
        Go = O.smoothed_gap(prob, xl[it - 1], yl[it - 1, :kml.m], p.xi)
        assert Go > 0
        assert abs(G[e] - Go) <= 2e-3 * abs(Go) + 1e-9, (it, G[e], Go)


def test_dual_start_must_lie_on_the_simplex(R, cuda, kml):
    s = R.Solver(kml.to(cuda), simplex_params(R))
    x = torch.zeros(kml.n, device=cuda)
    with pytest.raises(R.RapdbError):
        s.solve(x, torch.zeros(kml.m, device=cuda))
    with pytest.raises(R.RapdbError):
        s.solve(x, torch.tensor([0.5, 0.6, -0.1], device=cuda))
    s.close()
    with pytest.raises(R.RapdbError):
        R.Solver(kml.to(cuda), R.Params.default(dual_set=R.DUAL_SIMPLEX, dual_radius=0.0))


def test_kml_minmax_5000x8_bf16_full_size(R, cuda):
    """The paper's kernel-learning form at the n = 5000, m = 8 size in BF16
    storage with refinement, strongly convex with mu = 2 as in the paper:
    reaches rel KKT 1e-6, confirmed by the oracle's float64 residual at the
    solver's iterate."""
    data = W.config("C3m", device=cuda)
    p = simplex_params(R, mu=2.0, storage=1, refine=1, tol=1e-6, max_iter=20000, restart=R.RESTART_FIXED,
                       restart_period=200)
    s = R.Solver(data, p)
    x, y = start(data, cuda)
    info = s.solve(x, y)
    x64, y64 = s.solution_f64()
    s.close()
    assert info["status"] == R.OK and info["rel_kkt"] <= 1e-6, info
    prob = O.Problem.from_data(data.numpy())
    rel, _, _ = O.kkt_residual(prob, x64.cpu().numpy(), y64.cpu().numpy())
    assert rel <= 1e-6, rel
