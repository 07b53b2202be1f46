"""Symmetric block packing (pack_sym): the incremental trial pass read from the
upper block triangle of each Q_i, each off-diagonal 128 x 128 tile once for
its rows and, transposed, for its columns.

* the stand-alone packed pass against float64 products, under the bound its
  float32 arithmetic fixes: a row of W = Q v is a compensated sum over tiles
  of float32 partials; the longest float32 chain is the transposed one (8
  products per thread, then 16 warps in order), so each partial is within
  gamma_23 = 23 u / (1 - 23 u) of its exact value relative to the sum of
  |terms|, u = 2^-24; the compensated slot sum adds at most 2u of the sum
  (plus O(T^2 u^2) of the sum of |partials|), and the output one rounding;
* bit-for-bit reproducibility of the pass and of whole solves;
* the solver with packed trials against the FP64 oracle: the first iterates
  with a fixed step, full solves (yx, xy, fixed and adaptive restart), the
  smoothed gap computed through packed two-right-hand-side passes, the
  diagonal Q_0 with the simplex dual and a linear equality, BF16 storage with
  refinement, checkpoint / resume;
* sizes that leave a ragged last tile (n = 129, 200, 1000), one tile (128),
  and the full n = 4096, m = 50 workload on sampled rows and by the oracle's
  float64 KKT residual at the solver's iterate;
* FP8 storage with refinement and packing; BF16 and FP8 storage with adaptive
  restart, whose gap passes read the packed tiles after the precision switch;
* rejection of a non-symmetric Q and of levels 4 and 5 without packing.
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import quant as QZ
from paper_2605_29291_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
G23 = 23 * U32 / (1 - 23 * U32)


def oracle_params(R, p):
    restart = {R.RESTART_NONE: "none", R.RESTART_FIXED: "fixed", R.RESTART_GAP: "gap"}[p.restart]
    return O.Params(variant="yx" if p.variant == R.YX else "xy", c_nm=p.c_nm, backtracking=bool(p.backtracking),
                    mu=p.mu, c_alpha=p.c_alpha, c_beta=p.c_beta, delta=p.delta, eta=p.eta, tau_bar=p.tau_bar,
                    gamma0=p.gamma0, restart=restart, restart_period=p.restart_period,
                    restart_from_average=bool(p.restart_from_average), xi=p.xi, q=p.q, gap_first=p.gap_first,
                    gap_every=p.gap_every, max_iter=p.max_iter, max_trials=p.max_trials, kkt_every=p.kkt_every,
                    tol=p.tol, restart_warm_tau=bool(p.restart_warm_tau))


def packed(R, variant=0, **kw):
    return R.Params.default(variant, pack_sym=1, **kw)


def zeros(data, cuda):
    return (torch.zeros(data.n, dtype=torch.float32, device=cuda),
            torch.zeros(max(data.m, 1), dtype=torch.float32, device=cuda))


def stored_rows(data, si, rows, storage):
    """float64 rows of stored matrix si as the context stores it: the float32
    data, or its BF16 / Jacobi-scaled FP8 quantisation (the oracle's
    quantisers)."""
    dev = data.Q.device
    idx = torch.as_tensor(rows, device=dev)
    if storage == 0:
        return data.Q[si].index_select(0, idx).cpu().numpy().astype(np.float64)
    Qi = data.Q[si].cpu().numpy()
    if storage == 1:
        return QZ.bf16_round(Qi[rows]).astype(np.float64)
    codes, sc = QZ.fp8_jacobi_quantize(Qi)
    return QZ.fp8_dequantize(codes, sc)[rows]


def check_packed_pass(R, data, seed, rows=None, storage=0, vscale=None):
    """rapdb_packed_pass against float64 products on every (or the sampled)
    row of every stored matrix, under the gamma_23 bound; the dots against
    float64 sums of the same quantities; a second call bit-identical.  With
    BF16 / FP8 storage the pass reads the quantised tiles (the trials of the
    quantised level) and the products are those of the stored matrices; FP8
    adds one rounding per term (the pre-scaled s_k v_k) and one for the row
    scale."""
    dev = data.Q.device
    s = R.Solver(data, packed(R, storage=storage))
    n, M = data.n, int(data.Q.shape[0])
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    x = (data.lb + (data.ub - data.lb) * torch.rand(n, generator=g, device=dev)).contiguous()
    v = (1e-2 * torch.randn(n, generator=g, device=dev)).contiguous()
    if vscale is not None:   # one factor per 128-entry slice (the slices the tile kernels split)
        for b, f in enumerate(vscale):
            v[128 * b:128 * (b + 1)] *= f
    uold = torch.randn((M, n), generator=g, device=dev).contiguous()
    U, Wt, dots = s.packed_pass(x, v, uold)
    U2, W2, d2 = s.packed_pass(x, v, uold)
    s.close()
    assert torch.equal(U, U2) and torch.equal(Wt, W2) and torch.equal(dots, d2)
    rows = np.arange(n) if rows is None else rows
    x64, v64 = x.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    uo = uold.cpu().numpy().astype(np.float64)
    U, Wt, dots = U.cpu().numpy().astype(np.float64), Wt.cpu().numpy().astype(np.float64), dots.cpu().numpy()
    c = data.c.cpu().numpy().astype(np.float64)
    off = 0 if data.q0_kind == W.Q0_DENSE else 1
    gam = G23 if storage != 2 else G23 + 3 * U32
    for si in range(M):
        Qr = stored_rows(data, si, rows, storage)   # (k, n)
        w_ex = Qr @ v64
        aw = np.abs(Qr) @ np.abs(v64)
        u_ex = uo[si, rows] + w_ex
        # error of the unrounded w: partials + compensated slot sum (the
        # O(T^2 u^2) term and the float64 roundings are inside the 1e-3 slack)
        ew = (gam * aw + 2 * U32 * np.abs(w_ex)) * 1.001
        assert np.all(np.abs(Wt[si, rows] - w_ex) <= ew + U32 * np.abs(w_ex) * 1.001 + 1e-30), si
        assert np.all(np.abs(U[si, rows] - u_ex) <= ew + U32 * np.abs(u_ex) * 1.001 + 1e-30), si
        if len(rows) == n:
            # the dots use the unrounded float64 u and w
            i = si + off
            ax = np.abs(x64) @ ew + 1e-12 * (np.abs(x64) @ np.abs(u_ex))
            assert abs(dots[si, 0] - x64 @ u_ex) <= ax, si
            av = np.abs(v64) @ ew + 1e-12 * (np.abs(v64) @ np.abs(w_ex)) + 1e-300
            assert abs(dots[si, 1] - v64 @ w_ex) <= av, si
            t2 = v64 * uo[si]
            assert abs(dots[si, 2] - t2.sum()) <= 2.3e-16 * n * np.abs(t2).sum() + 1e-300
            for j, a in ((3, x64), (4, v64)):
                t = a * c[i]
                assert abs(dots[si, j] - t.sum()) <= 2.3e-16 * n * np.abs(t).sum() + 1e-300, (si, j)


@pytest.mark.parametrize("n,m", [(128, 2), (129, 3), (200, 10), (1000, 6)])
def test_packed_pass_matches_float64(R, cuda, n, m):
    data = W.random_qcqp(n, m, seed=n + m).to(cuda)
    check_packed_pass(R, data, seed=n)


def test_packed_pass_diag_q0(R, cuda):
    """Q_0 diagonal (not stored): the packed stored matrices are Q_1..Q_m."""
    data = W.kml_qcqp(120, 5, 8, seed=2).to(cuda)
    assert data.q0_kind == W.Q0_DIAG
    check_packed_pass(R, data, seed=3)


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("n,m", [(128, 2), (129, 3), (200, 10), (1000, 6)])
def test_quantised_packed_pass_matches_float64(R, cuda, storage, n, m):
    """The BF16 / FP8 tiles: products of the stored (quantised) matrices."""
    data = W.random_qcqp(n, m, seed=n + 3 * m).to(cuda)
    check_packed_pass(R, data, seed=n + 1, storage=storage)


@pytest.mark.parametrize("storage", [1, 2])
def test_quantised_packed_pass_slice_magnitudes(R, cuda, storage):
    """Right-hand-side slices of very different magnitudes, one of them all
    zero: the tensor-core path splits each 128-entry slice into pieces (FP8
    with a power-of-two scale per slice); the products still meet the
    float32 bound of the stored matrices."""
    data = W.random_qcqp(700, 4, seed=11).to(cuda)
    check_packed_pass(R, data, seed=6, storage=storage, vscale=[0.0, 1e-18, 1.0, 1e15, 3.0e-5, 7.0])


@pytest.mark.parametrize("storage", [1, 2])
def test_quantised_packed_pass_diag_q0(R, cuda, storage):
    data = W.kml_qcqp(120, 5, 8, seed=2).to(cuda)
    check_packed_pass(R, data, seed=4, storage=storage)


@pytest.mark.parametrize("variant", [0, 1])
def test_first_iterates_fixed_step(R, cuda, variant):
    c1 = W.config("C1")
    p = packed(R, variant, backtracking=0, tau_bar=0.05, tol=0.0, max_iter=50, restart=R.RESTART_NONE)
    s = R.Solver(c1.to(cuda), p)
    s.set_log(50)
    x, y = zeros(c1, cuda)
    info = s.solve(x, y)
    assert info["iters"] == 50
    xl = s.log["x"].cpu().numpy().astype(np.float64)
    yl = s.log["y"].cpu().numpy().astype(np.float64)
    s.close()
    r = O.rapdb(O.Problem.from_data(c1), p=oracle_params(R, p), keep_iterates=50)
    for k, (xo, lo) in enumerate(r.log["iterates"]):
        zo = np.concatenate([xo, lo])
        zg = np.concatenate([xl[k], yl[k, :c1.m]])
        assert np.linalg.norm(zg - zo) <= 1e-5 * max(1.0, np.linalg.norm(zo)), k


@pytest.mark.parametrize("variant,restart", [(0, 1), (0, 2), (1, 1), (1, 2)])
def test_full_solve_matches_oracle(R, cuda, variant, restart):
    c1 = W.config("C1")
    p = packed(R, variant, restart=restart, restart_period=200, tol=1e-6, max_iter=20000,
               gap_first=50 if variant == 0 else 100, gap_every=100)
    s = R.Solver(c1.to(cuda), p)
    s.set_log(30, iterates=False)
    x, y = zeros(c1, cuda)
    info = s.solve(x, y)
    assert info["status"] == R.OK and info["rel_kkt"] <= 1e-6, info
    prob = O.Problem.from_data(c1)
    r = O.rapdb(prob, p=oracle_params(R, p))
    assert r.status == 0
    np.testing.assert_array_equal(s.log["trials"].cpu().numpy()[:30], np.array(r.log["trials"][:30]))
    np.testing.assert_allclose(s.log["tau"].cpu().numpy()[:30], np.array(r.log["tau"][:30]), rtol=1e-9)
    x64, y64 = s.solution_f64()
    s.close()
    x64, y64 = x64.cpu().numpy(), y64.cpu().numpy()
    fo = prob.f(r.x)
    assert abs(info["obj"] - fo) <= 1e-5 * (1 + abs(fo))
    rel, _, _ = O.kkt_residual(prob, x64, y64)
    assert rel <= 1.1e-6, rel


@pytest.mark.parametrize("variant", [0, 1])
def test_smoothed_gap_through_packed_passes(R, cuda, variant):
    """The smoothed gap's two-right-hand-side passes read the packed tiles:
    G_xi at the logged iterates x^30, x^40 (fixed step) equals the oracle's
    exact G_xi within the subproblem's stopping bound, and the restarts fire
    as the oracle's rule says."""
    c1 = W.config("C1")
    kw = dict(backtracking=0, tau_bar=0.05, tol=0.0, max_iter=45, restart=R.RESTART_GAP, gap_first=30,
              gap_every=10)
    p = packed(R, variant, **kw)
    s = R.Solver(c1.to(cuda), p)
    s.set_log(50)
    x, y = zeros(c1, cuda)
    info = s.solve(x, y)
    assert info["iters"] == 45
    xl = s.log["x"].cpu().numpy().astype(np.float64)
    yl = s.log["y"].cpu().numpy().astype(np.float64)
    G = s.log["gap"].cpu().numpy().copy()
    s.close()
    prob = O.Problem.from_data(c1)
    for e, it in enumerate([30, 40]):
        Go = O.smoothed_gap(prob, xl[it - 1], yl[it - 1, :c1.m], p.xi)
        assert Go > 0
        assert abs(G[e] - Go) <= 2e-3 * abs(Go) + 1e-9, (it, G[e], Go)
    r = O.rapdb(prob, p=oracle_params(R, p))
    assert info["restarts"] == r.restarts


def test_packed_solve_is_deterministic_and_close_to_unpacked(R, cuda):
    data = W.random_qcqp(1000, 12, seed=9).to(cuda)
    out = []
    for _ in range(2):
        s = R.Solver(data, packed(R, restart=R.RESTART_GAP, tol=1e-6))
        x, y = zeros(data, cuda)
        info = s.solve(x, y)
        s.close()
        assert info["status"] == R.OK, info
        out.append((x, y, info))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    assert out[0][2]["iters"] == out[1][2]["iters"]
    s = R.Solver(data, R.Params.default(restart=R.RESTART_GAP, tol=1e-6))
    x, y = zeros(data, cuda)
    info = s.solve(x, y)
    s.close()
    assert info["status"] == R.OK
    prob = O.Problem.from_data(data.numpy())
    fp, fu = prob.f(out[0][0].cpu().numpy().astype(np.float64)), prob.f(x.cpu().numpy().astype(np.float64))
    assert abs(fp - fu) <= 1e-5 * (1 + abs(fu))


def test_checkpoint_resume_is_bit_identical(R, cuda):
    c1 = W.config("C1")
    full = packed(R, max_iter=300, tol=1e-9)
    s_full = R.Solver(c1.to(cuda), full)
    xf, yf = zeros(c1, cuda)
    i_full = s_full.solve(xf, yf)
    s_a = R.Solver(c1.to(cuda), packed(R, max_iter=137, tol=1e-9))
    xa, ya = zeros(c1, cuda)
    ia = s_a.solve(xa, ya)
    assert ia["status"] == R.ERR_MAXITER and ia["iters"] == 137
    s_b = R.Solver(c1.to(cuda), full)
    s_b.set_state(s_a.get_state())
    xb, yb = zeros(c1, cuda)
    ib = s_b.resume(xb, yb)
    assert ib["iters"] == i_full["iters"] and ib["trials"] == i_full["trials"]
    assert torch.equal(xb, xf) and torch.equal(yb, yf)
    for s in (s_full, s_a, s_b):
        s.close()


def test_simplex_dual_with_equality_and_diag_q0(R, cuda):
    """The kernel-learning min-max form (dual on the simplex, b'x = 0, Q_0
    diagonal) with packed trials against the oracle."""
    data = W.kml_minmax(200, 5, 3, seed=1, bias=True)
    p = packed(R, 0, dual_set=R.DUAL_SIMPLEX, dual_radius=1.0, restart=R.RESTART_FIXED, restart_period=200,
               tol=1e-6, max_iter=30000)
    s = R.Solver(data.to(cuda), p)
    x = torch.zeros(data.n, dtype=torch.float32, device=cuda)
    y = torch.zeros(s.m, dtype=torch.float32, device=cuda)
    y[:data.m] = 1.0 / data.m
    info = s.solve(x, y)
    x64, y64 = s.solution_f64()
    s.close()
    assert info["status"] == R.OK and info["rel_kkt"] <= 1e-6, info
    prob = O.Problem.from_data(data)
    r = O.rapdb(prob, p=oracle_params(R, p))
    assert r.status == 0
    xg, yg = x64.cpu().numpy(), y64.cpu().numpy()
    fo = prob.phi(r.x, r.lam)
    assert abs(prob.phi(xg, yg) - fo) <= 1e-5 * (1 + abs(fo))
    rel, _, _ = O.kkt_residual(prob, xg, yg)
    assert rel <= 1.1e-6, rel


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("case", ["kml", "random"])
def test_quantised_level_solve_meets_tolerance(R, cuda, storage, case):
    """BF16 / FP8 storage with refinement and packing: the trials add the
    increments Q~ d of the quantised tiles to float32 compensated products,
    re-anchored at the check every 64 accepted iterations; a stall there
    that the storage explains switches to the float32 tiles.  The solve ends
    at rel KKT 1e-6 of the
    float32 problem by the oracle's float64 residual, whether or not it
    switched (switch_iter says when it did)."""
    data = W.kml_qcqp(200, 6, 8, seed=4 + storage) if case == "kml" else W.random_qcqp(300, 8, seed=7)
    p = packed(R, storage=storage, refine=1, tol=1e-6, restart_period=100, max_iter=20000)
    s = R.Solver(data.to(cuda), p)
    x, y = zeros(data, cuda)
    info = s.solve(x, y)
    x64, y64 = s.solution_f64()
    s.close()
    assert info["status"] == R.OK, info
    assert (info["switch_iter"] >= 0) == (info["precision_switches"] >= 1), info
    rel, _, _ = O.kkt_residual(O.Problem.from_data(data), x64.cpu().numpy(), y64.cpu().numpy())
    assert rel <= 1.1e-6, rel


@pytest.mark.parametrize("storage", [1, 2])
def test_quantised_storage_adaptive_restart_packed_gap(R, cuda, storage):
    """BF16 / FP8 storage with refinement, adaptive restart and packing: the
    smoothed gap's passes read the packed float32 tiles, the trials the
    quantised ones; the solve ends at rel KKT 1e-6 by the oracle's float64
    residual."""
    data = W.kml_qcqp(200, 6, 8, seed=4)
    p = packed(R, storage=storage, refine=1, tol=1e-6, restart=R.RESTART_GAP, gap_first=20, gap_every=20,
               restart_period=100, max_iter=20000)
    s = R.Solver(data.to(cuda), p)
    x, y = zeros(data, cuda)
    info = s.solve(x, y)
    x64, y64 = s.solution_f64()
    s.close()
    assert info["status"] == R.OK, info
    assert info["passes"] > info["trials"] + 20, info          # gap passes ran
    rel, _, _ = O.kkt_residual(O.Problem.from_data(data), x64.cpu().numpy(), y64.cpu().numpy())
    assert rel <= 1.1e-6, rel


def test_non_symmetric_q_rejected(R, cuda):
    data = W.random_qcqp(150, 3, seed=1)
    data.Q[2, 7, 140] += np.float32(1e-3)
    with pytest.raises(R.RapdbError):
        R.Solver(data.to(cuda), packed(R))
    # the same data without packing is accepted
    R.Solver(data.to(cuda), R.Params.default()).close()


def test_time_pass_level_4(R, cuda):
    data = W.random_qcqp(300, 4, seed=2).to(cuda)
    s = R.Solver(data, packed(R))
    ms, b = s.time_pass(reps=3, level=4)
    T = (300 + 127) // 128
    assert ms > 0 and b == 5 * T * (T + 1) // 2 * 128 * 128 * 4
    ms5, b5 = s.time_pass(reps=3, level=5)
    assert ms5 > 0 and b5 == b
    ms3, b3 = s.time_pass(reps=3, level=3)
    assert b3 == 5 * 300 * 300 * 4
    s.close()
    with pytest.raises(R.RapdbError):
        s.time_pass(reps=1, level=6)      # a float32 context has no quantised tiles
    s.close()
    s = R.Solver(data, R.Params.default())
    for lv in (4, 5):
        with pytest.raises(R.RapdbError):
            s.time_pass(reps=1, level=lv)
    s.close()
    for storage, eb in ((1, 2), (2, 1)):
        s = R.Solver(data, packed(R, storage=storage))
        ms6, b6 = s.time_pass(reps=3, level=6)
        ms7, b7 = s.time_pass(reps=3, level=7)
        q = 5 * T * (T + 1) // 2 * 128 * 128 * eb + (5 * 300 * 4 if storage == 2 else 0)
        assert ms6 > 0 and ms7 > 0 and b6 == q and b7 == q
        s.close()


# ---------------------------------------------------------------------------
# Full size: dense random QCQP n = 4096, m = 50 (the benchmark's workload)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def c2(cuda):
    d = W.config("C2", device=cuda)
    yield d
    del d
    torch.cuda.empty_cache()


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_dense_4096x50_packed_pass_sampled_rows(R, c2, storage):
    rng = np.random.default_rng(5)
    rows = np.sort(np.concatenate([[0, 127, 128, c2.n - 1], rng.choice(np.arange(129, c2.n - 1), 36, False)]))
    check_packed_pass(R, c2, seed=5, rows=rows, storage=storage)


def test_dense_4096x50_packed_solve_meets_tolerance(R, cuda, c2):
    p = packed(R, c_nm=1, restart=R.RESTART_GAP, gap_first=50, gap_every=500, restart_period=200, tol=1e-6,
               max_iter=50000, time_limit_s=300.0)
    s = R.Solver(c2, p)
    x, y = zeros(c2, cuda)
    info = s.solve(x, y)
    x64, y64 = s.solution_f64()
    s.close()
    assert info["status"] == R.OK and info["rel_kkt"] <= 1e-6, info
    prob = O.Problem.from_data(c2.numpy())
    x64, y64 = x64.cpu().numpy(), y64.cpu().numpy()
    assert np.all(x64 >= prob.lb) and np.all(x64 <= prob.ub) and np.all(y64 >= 0)
    rel, _, _ = O.kkt_residual(prob, x64, y64)
    assert rel <= 1e-6, rel
