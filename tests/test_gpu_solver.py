"""The device-resident rAPDB loop against the FP64 oracle.

* fixed step, backtracking off: the first 50 iterates agree to
  ||z_gpu - z_oracle|| <= 1e-5 max(1, ||z_oracle||)  (z = (x, y));
* with backtracking: the accept/reject pattern of the first iterations, the
  final objective to rel 1e-5 and the relative KKT residual <= 1e-6, checked
  again by the oracle's own FP64 residual at the GPU's point;
* closed forms (ball constraint, interior PD QP), ragged sizes, diagonal and
  zero Q_0, quantised storage with float32 refinement, restarts from the
  average, checkpoint / resume, batching and the error statuses.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2605_29291_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def gpu_vecs(data, cuda, x0=None, y0=None):
    x = torch.zeros(data.n, dtype=torch.float32, device=cuda) if x0 is None else \
        torch.as_tensor(np.asarray(x0, np.float32)).to(cuda)
    y = torch.zeros(max(data.m, 1), dtype=torch.float32, device=cuda) if y0 is None else \
        torch.as_tensor(np.asarray(y0, np.float32)).to(cuda)
    return x, y


def oracle_params(R, p, **kw):
    """Oracle Params from the library's Params (same numbers)."""
    restart = {R.RESTART_NONE: "none", R.RESTART_FIXED: "fixed", R.RESTART_GAP: "gap"}[p.restart]
    return O.Params(variant="yx" if p.variant == R.YX else "xy", c_nm=p.c_nm, backtracking=bool(p.backtracking),
                    mu=p.mu, c_alpha=p.c_alpha, c_beta=p.c_beta, delta=p.delta, eta=p.eta, tau_bar=p.tau_bar,
                    gamma0=p.gamma0, restart=restart, restart_period=p.restart_period,
                    restart_from_average=bool(p.restart_from_average), xi=p.xi, q=p.q, gap_first=p.gap_first,
                    gap_every=p.gap_every, max_iter=p.max_iter, max_trials=p.max_trials, kkt_every=p.kkt_every,
                    tol=p.tol, restart_warm_tau=bool(p.restart_warm_tau), **kw)


@pytest.fixture(scope="module")
def c1():
    return W.config("C1")


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("restart_avg", [0, 1])
def test_first_50_iterates_fixed_step(R, cuda, c1, variant, restart_avg):
    p = R.Params.default(variant, backtracking=0, tau_bar=0.05, tol=0.0, max_iter=50,
                         restart=R.RESTART_FIXED if restart_avg else R.RESTART_NONE, restart_period=20,
                         restart_from_average=restart_avg)
    s = R.Solver(c1.to(cuda), p)
    s.set_log(50)
    x, y = gpu_vecs(c1, cuda)
    info = s.solve(x, y)
    assert info["status"] == R.ERR_MAXITER and info["iters"] == 50
    xl = s.log["x"].cpu().numpy().astype(np.float64)
    yl = s.log["y"].cpu().numpy().astype(np.float64)
    prob = O.Problem.from_data(c1)
    r = O.rapdb(prob, p=oracle_params(R, p), keep_iterates=50)
    assert len(r.log["iterates"]) == 50
    for k, (xo, lo) in enumerate(r.log["iterates"]):
        zo = np.concatenate([xo, lo])
        zg = np.concatenate([xl[k], yl[k, :c1.m]])
        assert np.linalg.norm(zg - zo) <= 1e-5 * max(1.0, np.linalg.norm(zo)), k
    if restart_avg:
        assert info["restarts"] == r.restarts == 2
    s.close()


@pytest.mark.parametrize("variant,c_nm", [(0, 1), (0, 0), (1, 1)])
def test_full_solve_matches_oracle(R, cuda, c1, variant, c_nm):
    p = R.Params.default(variant, c_nm=c_nm, restart_period=200, tol=1e-6, max_iter=20000)
    s = R.Solver(c1.to(cuda), p)
    s.set_log(30, iterates=False)
    x, y = gpu_vecs(c1, cuda)
    info = s.solve(x, y)
    assert info["status"] == R.OK, info
    assert info["rel_kkt"] <= 1e-6
    prob = O.Problem.from_data(c1)
    r = O.rapdb(prob, p=oracle_params(R, p))
    assert r.status == 0
    # same decisions over the first iterations
    np.testing.assert_array_equal(s.log["trials"].cpu().numpy()[:30], np.array(r.log["trials"][:30]))
    np.testing.assert_allclose(s.log["tau"].cpu().numpy()[:30], np.array(r.log["tau"][:30]), rtol=1e-9)
    xg = x.cpu().numpy().astype(np.float64)
    yg = y.cpu().numpy().astype(np.float64)[:c1.m]
    fo = prob.f(r.x)
    assert abs(prob.f(xg) - fo) <= 1e-5 * (1 + abs(fo))
    assert abs(info["obj"] - fo) <= 1e-5 * (1 + abs(fo))
    rel, _, _ = O.kkt_residual(prob, xg, yg)
    assert rel <= 2e-6
    # the library's stand-alone KKT residual (compensated products) agrees
    # with the oracle's float64 residual at the same float32 point
    rel_lib, rs_lib, rf_lib = s.kkt_residual(x, y)
    assert abs(rel_lib - rel) <= 1e-3 * rel + 1e-12
    assert abs(info["iters"] - r.iters) <= max(10, 0.1 * r.iters)
    s.close()


def test_solve_is_deterministic(R, cuda, c1):
    s = R.Solver(c1.to(cuda))
    x1, y1 = gpu_vecs(c1, cuda)
    i1 = s.solve(x1, y1)
    x2, y2 = gpu_vecs(c1, cuda)
    i2 = s.solve(x2, y2)
    assert torch.equal(x1, x2) and torch.equal(y1, y2)
    assert i1["iters"] == i2["iters"] and i1["trials"] == i2["trials"]
    s.close()


@pytest.mark.parametrize("q0_kind", [W.Q0_DENSE, W.Q0_ZERO])
@pytest.mark.parametrize("variant", [0, 1])
def test_ball_closed_form(R, cuda, q0_kind, variant):
    """min c'x s.t. ||x||^2 <= rho^2: x* = -rho c/||c||, y* = ||c||/(2 rho)."""
    rng = np.random.default_rng(11)
    cvec = rng.standard_normal(37).astype(np.float32)
    rho = 2.0
    data = W.ball_qcqp(cvec, rho)
    if q0_kind == W.Q0_ZERO:
        data = W.QCQPData(data.n, data.m, data.Q[1:].copy(), data.c, data.d, data.lb, data.ub, W.Q0_ZERO)
    p = R.Params.default(variant, tol=1e-7, max_iter=50000)
    s = R.Solver(data.to(cuda), p)
    x, y = gpu_vecs(data, cuda)
    info = s.solve(x, y)
    assert info["status"] == R.OK, info
    c64 = cvec.astype(np.float64)
    np.testing.assert_allclose(x.cpu().numpy(), -rho * c64 / np.linalg.norm(c64), atol=2e-4)
    np.testing.assert_allclose(y.cpu().numpy()[0], np.linalg.norm(c64) / (2 * rho), rtol=2e-4)
    s.close()


def test_interior_pd_qp_closed_form(R, cuda):
    """m = 0, Q_0 PD, interior minimiser: x* = -Q_0^{-1} c_0."""
    rng = np.random.default_rng(5)
    n = 40
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Q0 = ((U * rng.uniform(1.0, 5.0, n)) @ U.T).astype(np.float32)
    Q0 = ((Q0 + Q0.T) * np.float32(0.5)).astype(np.float32)
    c = np.zeros((1, n), np.float32)
    c[0] = rng.standard_normal(n)
    data = W.QCQPData(n, 0, Q0[None], c, np.zeros(0, np.float32), np.full(n, -10, np.float32),
                      np.full(n, 10, np.float32))
    s = R.Solver(data.to(cuda), R.Params.default(tol=1e-6))
    x, y = gpu_vecs(data, cuda)
    info = s.solve(x, y)
    assert info["status"] == R.OK, info
    xs = -np.linalg.solve(Q0.astype(np.float64), c[0].astype(np.float64))
    np.testing.assert_allclose(x.cpu().numpy(), xs, atol=1e-5 * (1 + np.abs(xs).max()))
    s.close()


@pytest.mark.parametrize("n,m", [(203, 3), (61, 5), (300, 4)])
def test_ragged_sizes_match_oracle(R, cuda, n, m):
    data = W.random_qcqp(n, m, seed=n)
    p = R.Params.default(tol=1e-6, max_iter=20000)
    s = R.Solver(data.to(cuda), p)
    s.set_log(20, iterates=False)
    x, y = gpu_vecs(data, cuda)
    info = s.solve(x, y)
    assert info["status"] == R.OK and info["rel_kkt"] <= 1e-6
    prob = O.Problem.from_data(data)
    r = O.rapdb(prob, p=oracle_params(R, p))
    np.testing.assert_array_equal(s.log["trials"].cpu().numpy()[:20], np.array(r.log["trials"][:20]))
    fo = prob.f(r.x)
    assert abs(info["obj"] - fo) <= 1e-5 * (1 + abs(fo))
    s.close()


def test_objective_and_infeasibility_logs(R, cuda):
    """The logged f(x^{k+1}) and mean_i max(g_i(x^{k+1}), 0) -- the paper's
    termination measure for random QCQPs -- equal the oracle's f and g at the
    logged iterates (float32 copies of the float64 iterates, hence the
    tolerance scaled by |x| |grad|)."""
    data = W.paper_random_qcqp(200, 5, seed=3)
    p = R.Params.default(R.YX, tol=1e-12, max_iter=60, restart=R.RESTART_FIXED, restart_period=400)
    s = R.Solver(data.to(cuda), p)
    s.set_log(60)
    x, y = gpu_vecs(data, cuda)
    info = s.solve(x, y, check=False)
    assert info["iters"] == 60
    xl = s.log["x"].cpu().numpy().astype(np.float64)
    ob = s.log["obj"].cpu().numpy()
    inf = s.log["infeas"].cpu().numpy()
    s.close()
    prob = O.Problem.from_data(data)
    for e in range(60):
        xe = xl[e]
        g = prob.g(xe)
        f = prob.f(xe)
        sc_f = 1.0 + np.linalg.norm(xe) * (np.linalg.norm(prob.Q[0] @ xe) + np.linalg.norm(prob.c[0]))
        assert abs(ob[e] - f) <= 1e-6 * sc_f, (e, ob[e], f)
        sc_g = 1.0 + max(np.linalg.norm(xe) * (np.linalg.norm(prob.Q[i] @ xe) + np.linalg.norm(prob.c[i]))
                         for i in range(1, prob.m + 1))
        assert abs(inf[e] - np.mean(np.maximum(g, 0.0))) <= 1e-6 * sc_g, e


def test_kml_diag_q0_matches_oracle(R, cuda):
    data = W.kml_qcqp(120, 5, 8, seed=2)
    p = R.Params.default(tol=1e-6, restart_period=200)
    s = R.Solver(data.to(cuda), p)
    x, y = gpu_vecs(data, cuda)
    info = s.solve(x, y)
    assert info["status"] == R.OK, info
    prob = O.Problem.from_data(data)
    r = O.rapdb(prob, p=oracle_params(R, p))
    fo = prob.f(r.x)
    assert abs(info["obj"] - fo) <= 1e-5 * (1 + abs(fo))
    rel, _, _ = O.kkt_residual(prob, x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64))
    assert rel <= 2e-6
    s.close()


@pytest.mark.parametrize("storage", [1, 2])
def test_quantised_storage_with_refinement(R, cuda, storage):
    """BF16 / FP8 storage, switched to the float32 Q (compensated products)
    when a precision check finds the true KKT residual stalled or dominated
    by the storage error: ends at rel KKT <= 1e-6 of the float32 problem."""
    data = W.kml_qcqp(200, 6, 8, seed=4)
    p = R.Params.default(storage=storage, refine=1, tol=1e-6, restart_period=100)
    s = R.Solver(data.to(cuda), p)
    x, y = gpu_vecs(data, cuda)
    info = s.solve(x, y)
    assert info["status"] == R.OK, info
    assert info["precision_switches"] >= 1
    prob = O.Problem.from_data(data)
    rel, _, _ = O.kkt_residual(prob, x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64))
    assert rel <= 2e-6
    # the stand-alone residual at the returned float32 point matches the oracle's
    rel_lib, _, _ = s.kkt_residual(x, y)
    assert abs(rel_lib - rel) <= 1e-3 * rel + 1e-12
    # the solver's own float64 iterate meets the tolerance
    x64, y64 = s.solution_f64()
    rel64, _, _ = O.kkt_residual(prob, x64.cpu().numpy(), y64.cpu().numpy())
    assert rel64 <= 1.1e-6
    r = O.rapdb(prob, p=O.default_params("yx", tol=1e-7, restart_period=100))
    fo = prob.f(r.x)
    assert abs(prob.f(x.cpu().numpy().astype(np.float64)) - fo) <= 1e-5 * (1 + abs(fo))
    s.close()


def test_checkpoint_resume_is_bit_identical(R, cuda, c1):
    # one tile for all three contexts: tiles with different rows per warp
    # combine the products in different (each fixed) orders
    tile = dict(rows_per_block=64, pass_variant=0)
    full = R.Params.default(max_iter=300, tol=1e-9, **tile)
    s_full = R.Solver(c1.to(cuda), full)
    xf, yf = gpu_vecs(c1, cuda)
    i_full = s_full.solve(xf, yf)
    part = R.Params.default(max_iter=137, tol=1e-9, **tile)
    s_a = R.Solver(c1.to(cuda), part)
    xa, ya = gpu_vecs(c1, cuda)
    ia = s_a.solve(xa, ya)
    assert ia["status"] == R.ERR_MAXITER and ia["iters"] == 137
    blob = s_a.get_state()
    s_b = R.Solver(c1.to(cuda), full)
    s_b.set_state(blob)
    xb, yb = gpu_vecs(c1, cuda)
    ib = s_b.resume(xb, yb)
    assert ib["iters"] == i_full["iters"] and ib["trials"] == i_full["trials"]
    assert torch.equal(xb, xf) and torch.equal(yb, yf)
    for s in (s_full, s_a, s_b):
        s.close()


def test_batched_matches_single(R, cuda):
    datas = W.batched_random_qcqp(12, seed=3, n_lo=32, n_hi=300, m_lo=1, m_hi=8)
    p = R.Params.default(tol=1e-6)
    devs = [d.to(cuda) for d in datas]
    bs = R.BatchedSolver(devs, p)
    xs = [torch.zeros(d.n, device=cuda) for d in datas]
    ys = [torch.zeros(max(d.m, 1), device=cuda) for d in datas]
    infos = bs.solve(xs, ys)
    # the autotuner's tiles: one variant for the batch, rows per block per size class
    tiles = [bs.tile(b) for b in range(len(datas))]
    assert len({t["variant"] for t in tiles}) == 1
    assert all(t["rows_per_block"] in (32, 64, 128) for t in tiles)
    by_class = {}
    for d, t in zip(datas, tiles):
        by_class.setdefault(int(np.ceil(np.log2(d.n))), set()).add(t["rows_per_block"])
    assert all(len(v) == 1 for v in by_class.values())
    # a single-instance context with the instance's tile performs the same
    # floating-point operations
    for d, dv, xb, yb, ib, t in zip(datas, devs, xs, ys, infos, tiles):
        assert ib["status"] == R.OK and ib["rel_kkt"] <= 1e-6
        p1 = R.Params.default(tol=1e-6, rows_per_block=t["rows_per_block"], pass_variant=t["variant"])
        s = R.Solver(dv, p1)
        x, y = gpu_vecs(d, cuda)
        i1 = s.solve(x, y)
        assert i1["iters"] == ib["iters"] and i1["trials"] == ib["trials"]
        assert torch.equal(x, xb) and torch.equal(y[:d.m], yb[:d.m])
        s.close()
    bs.close()


def test_status_codes(R, cuda, c1):
    s = R.Solver(c1.to(cuda), R.Params.default(max_iter=5, tol=0.0))
    x, y = gpu_vecs(c1, cuda)
    assert s.solve(x, y)["status"] == R.ERR_MAXITER
    s.close()
    s = R.Solver(c1.to(cuda), R.Params.default(time_limit_s=1e-9, tol=0.0, max_iter=10 ** 6))
    x, y = gpu_vecs(c1, cuda)
    assert s.solve(x, y)["status"] == R.ERR_TIMEOUT
    s.close()
    # x0 outside the box, y0 negative
    s = R.Solver(c1.to(cuda))
    x, y = gpu_vecs(c1, cuda)
    x[0] = 11.0
    with pytest.raises(R.RapdbError):
        s.solve(x, y)
    x, y = gpu_vecs(c1, cuda)
    y[0] = -1.0
    with pytest.raises(R.RapdbError):
        s.solve(x, y)
    s.close()


@pytest.mark.parametrize("fault", ["nan", "box", "diag"])
def test_invalid_data_rejected(R, cuda, fault):
    data = W.random_qcqp(40, 2, seed=1)
    h = data.numpy()
    Q, lb = h.Q.copy(), h.lb.copy()
    if fault == "nan":
        Q[1, 3, 5] = np.nan
    elif fault == "box":
        lb[7] = 20.0
    else:
        Q[2, 4, 4] = -1.0
    bad = W.QCQPData(40, 2, Q, h.c, h.d, lb, h.ub)
    with pytest.raises(R.RapdbError) as e:
        R.Solver(bad.to(cuda))
    assert e.value.status == R.ERR_INVALID


def test_kkt_residual_at_random_points(R, cuda, c1):
    s = R.Solver(c1.to(cuda))
    prob = O.Problem.from_data(c1)
    rng = np.random.default_rng(4)
    for _ in range(3):
        x = rng.uniform(-1, 1, c1.n).astype(np.float32)
        x[:5] = 10.0
        y = rng.uniform(0, 1, c1.m).astype(np.float32)
        y[:2] = 0.0
        rel, rs, rf = s.kkt_residual(torch.from_numpy(x).to(cuda), torch.from_numpy(y).to(cuda))
        ro, rso, rfo = O.kkt_residual(prob, x.astype(np.float64), y.astype(np.float64))
        np.testing.assert_allclose([rel, rs, rf], [ro, rso, rfo], rtol=1e-5)
    s.close()


@pytest.mark.parametrize("variant", [0, 1])
def test_smoothed_gap_matches_oracle_at_logged_iterates(R, cuda, c1, variant):
    """Adaptive restart (eq. ada_restart): the device's G_xi at iterates x^30,
    x^40 (fixed step, so both sides are at the same point) equals the oracle's
    exact G_xi (y-part closed form, x-part an exact box QP) within the
    subproblem's stopping bound (1e-3 of G)."""
    p = R.Params.default(variant, backtracking=0, tau_bar=0.05, tol=0.0, max_iter=45, restart=R.RESTART_GAP,
                         gap_first=30, gap_every=10)
    s = R.Solver(c1.to(cuda), p)
    s.set_log(50)
    x, y = gpu_vecs(c1, cuda)
    info = s.solve(x, y)
    assert info["iters"] == 45
    xl = s.log["x"].cpu().numpy().astype(np.float64)
    yl = s.log["y"].cpu().numpy().astype(np.float64)
    G = s.log["gap"].cpu().numpy()
    prob = O.Problem.from_data(c1)
    for e, it in enumerate([30, 40]):
        Go = O.smoothed_gap(prob, xl[it - 1], yl[it - 1, :c1.m], p.xi)
        assert Go > 0
        # the device stops the x-subproblem once its error bound is below 1e-3 of the gap
        assert abs(G[e] - Go) <= 2e-3 * abs(Go) + 1e-9, (it, G[e], Go)
    # the restart fired exactly when the oracle's rule says so
    r = O.rapdb(prob, p=oracle_params(R, p))
    assert info["restarts"] == r.restarts
    s.close()


def test_adaptive_restart_full_solve(R, cuda, c1):
    p = R.Params.default(R.YX, restart=R.RESTART_GAP, gap_first=50, gap_every=100, tol=1e-6, max_iter=20000)
    s = R.Solver(c1.to(cuda), p)
    s.set_log(64, iterates=False)
    x, y = gpu_vecs(c1, cuda)
    info = s.solve(x, y)
    assert info["status"] == R.OK, info
    prob = O.Problem.from_data(c1)
    r = O.rapdb(prob, p=oracle_params(R, p))
    assert r.status == 0
    fo = prob.f(r.x)
    assert abs(info["obj"] - fo) <= 1e-5 * (1 + abs(fo))
    G = s.log["gap"].cpu().numpy()
    Go = [g for (_, g, _) in r.log["gap"]]
    # the first evaluation (k = 50) happens before the trajectories part
    assert abs(G[0] - Go[0]) <= 3e-3 * abs(Go[0])
    # (the precision switch of the refinement keeps the iteration's state, so
    # it adds no restart; the trajectories still part after it)
    assert abs(info["restarts"] - r.restarts) <= 1
    # each pass of the gap evaluation is counted; the solve still ends near the oracle
    assert info["passes"] > info["trials"]
    s.close()


def test_compensated_refinement_breaks_float32_floor(R, cuda):
    """n = 1024, m = 50: plain float32 products stall near rel KKT 1.3e-6 on
    this instance (the Lagrangian gradient cancels the per-constraint
    products' rounding).  With refinement the solver runs compensated
    (double-float) products from the start, needs no precision switch, and
    reaches 2e-7, confirmed by the oracle's float64 residual at the returned
    point."""
    data = W.random_qcqp(1024, 50, rows=512, seed=0)
    p = R.Params.default(tol=2e-7, max_iter=6000, refine=1)
    s = R.Solver(data.to(cuda), p)
    x, y = gpu_vecs(data, cuda)
    info = s.solve(x, y)
    assert info["status"] == R.OK, info
    assert info["precision_switches"] == 0 and info["rel_kkt"] <= 2e-7
    prob = O.Problem.from_data(data)
    x64, y64 = s.solution_f64()
    rel, _, _ = O.kkt_residual(prob, x64.cpu().numpy(), y64.cpu().numpy())
    assert rel <= 3e-7
    # the float32 copy returned by rapdb_solve is the same point rounded
    np.testing.assert_array_equal(x.cpu().numpy(), x64.cpu().numpy().astype(np.float32))
    s.close()
    p0 = R.Params.default(tol=2e-7, max_iter=3000, refine=0)
    s = R.Solver(data.to(cuda), p0)
    x, y = gpu_vecs(data, cuda)
    info0 = s.solve(x, y)
    assert info0["status"] == R.ERR_MAXITER      # the float32 floor without refinement
    s.close()


MODES = [(v, cnm, rs) for v in (0, 1) for cnm in (0, 1) for rs in ("none", "fixed", "gap")]


@pytest.mark.parametrize("variant,c_nm,restart", MODES)
def test_method_modes_match_oracle(R, cuda, variant, c_nm, restart):
    """Every combination of yx/xy, monotone/non-monotone step rule and
    none/fixed/adaptive restart reaches the oracle's objective and a float64
    residual <= 1e-6 at the solver's iterate."""
    data = W.random_qcqp(150, 4, rows=75, seed=21)
    rmode = {"none": R.RESTART_NONE, "fixed": R.RESTART_FIXED, "gap": R.RESTART_GAP}[restart]
    p = R.Params.default(variant, c_nm=c_nm, restart=rmode, restart_period=100, gap_first=40, gap_every=100,
                         tol=1e-6, max_iter=30000)
    s = R.Solver(data.to(cuda), p)
    x, y = gpu_vecs(data, cuda)
    info = s.solve(x, y)
    assert info["status"] == R.OK, info
    prob = O.Problem.from_data(data)
    x64, y64 = s.solution_f64()
    rel, _, _ = O.kkt_residual(prob, x64.cpu().numpy(), y64.cpu().numpy())
    assert rel <= 1.1e-6
    r = O.rapdb(prob, p=O.default_params("yx", tol=1e-8, max_iter=50000))
    fo = prob.f(r.x)
    assert abs(prob.f(x64.cpu().numpy()) - fo) <= 1e-5 * (1 + abs(fo))
    s.close()


def test_bf16_with_adaptive_restart(R, cuda):
    data = W.random_qcqp(300, 6, rows=150, seed=6)
    p = R.Params.default(storage=R.BF16, restart=R.RESTART_GAP, gap_first=50, gap_every=150, tol=1e-6,
                         max_iter=30000)
    s = R.Solver(data.to(cuda), p)
    x, y = gpu_vecs(data, cuda)
    info = s.solve(x, y)
    assert info["status"] == R.OK and info["precision_switches"] >= 1, info
    prob = O.Problem.from_data(data)
    x64, y64 = s.solution_f64()
    rel, _, _ = O.kkt_residual(prob, x64.cpu().numpy(), y64.cpu().numpy())
    assert rel <= 1.1e-6
    s.close()


def test_batched_xy_adaptive_matches_single(R, cuda):
    datas = W.batched_random_qcqp(6, seed=8, n_lo=40, n_hi=200, m_lo=1, m_hi=5)
    p = R.Params.default(R.XY, restart=R.RESTART_GAP, gap_first=30, gap_every=100, tol=1e-6, max_iter=30000,
                         rows_per_block=64, pass_variant=6)
    devs = [d.to(cuda) for d in datas]
    bs = R.BatchedSolver(devs, p)
    xs = [torch.zeros(d.n, device=cuda) for d in datas]
    ys = [torch.zeros(max(d.m, 1), device=cuda) for d in datas]
    infos = bs.solve(xs, ys)
    for d, dv, xb, yb, ib in zip(datas, devs, xs, ys, infos):
        assert ib["status"] == R.OK, ib
        s = R.Solver(dv, p)
        x, y = gpu_vecs(d, cuda)
        i1 = s.solve(x, y)
        assert i1["iters"] == ib["iters"] and i1["restarts"] == ib["restarts"]
        assert torch.equal(x, xb)
        s.close()
    bs.close()


@pytest.mark.parametrize("variant", [0, 1])
def test_warm_started_tau_across_restarts_matches_oracle(R, cuda, c1, variant):
    """With restart_warm_tau a restart starts from the last accepted tau: the
    same accept/reject pattern and step sizes as the oracle across the
    restarts at k = 40, 80, and the same solution."""
    p = R.Params.default(variant, restart=R.RESTART_FIXED, restart_period=40, restart_warm_tau=1, tol=1e-6,
                         max_iter=20000)
    s = R.Solver(c1.to(cuda), p)
    s.set_log(120, iterates=False)
    x, y = gpu_vecs(c1, cuda)
    info = s.solve(x, y)
    assert info["status"] == R.OK, info
    prob = O.Problem.from_data(c1)
    r = O.rapdb(prob, p=oracle_params(R, p))
    assert r.status == 0
    k = min(120, info["iters"], r.iters)
    np.testing.assert_array_equal(s.log["trials"].cpu().numpy()[:k], np.array(r.log["trials"][:k]))
    np.testing.assert_allclose(s.log["tau"].cpu().numpy()[:k], np.array(r.log["tau"][:k]), rtol=1e-9)
    fo = prob.f(r.x)
    assert abs(info["obj"] - fo) <= 1e-5 * (1 + abs(fo))
    s.close()
