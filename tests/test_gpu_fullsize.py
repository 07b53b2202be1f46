"""Parity at the full sizes of the named workloads, in the launch configuration
the benchmark times (autotuned tiles, the benchmark's solver parameters):

  * dense random QCQP n = 4096, m = 50, float32 storage (3.42 GB stack);
  * kernel-learning epigraph QCQP n = 5000 (+1), m = 8, bfloat16 storage;
  * 256 random QCQPs of uneven n (64..1024) and m (2..32) in one batched loop;
  * kernel-learning epigraph QCQP n = 16000 (+1), m = 20, Jacobi-scaled FP8
    storage (5.1 GB of codes over a 20.5 GB float32 stack).

The oracle cannot run these whole, so the checks are on sampled outputs it
computes one by one (rows of every Q_i x and Q_i v, columns of the stored
matrices, code by code) and on properties that hold at any size (the
float64 KKT residual of the oracle at the solver's result, box and sign
feasibility, the reduction dots against the kernel's own products)."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import quant as QZ
from paper_2605_29291_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N_SAMPLE = 40


def bench_params(R, variant=None, **kw):
    """The benchmark's solver parameters: yx, non-monotone steps, adaptive
    restart (first gap evaluation at k = 50, then every 500), refinement on.
    The xy variant takes its own defaults (first gap evaluation at k = 100)."""
    variant = R.YX if variant is None else variant
    base = dict(c_nm=1, restart=R.RESTART_GAP, gap_first=50 if variant == R.YX else 100, gap_every=500,
                restart_period=200, tol=1e-6, max_iter=50000, time_limit_s=300.0, refine=1)
    base.update(kw)
    return R.Params.default(variant, **base)


def sample_rows(n, seed):
    """Sampled row indices: the first and last rows (the ragged tail of the
    last row block) and random rows in between."""
    rng = np.random.default_rng(seed)
    mid = rng.choice(np.arange(1, n - 1), size=N_SAMPLE - 2, replace=False)
    return np.sort(np.concatenate([[0, n - 1], mid]))


def stored_rows(data, storage, rows):
    """float64 rows `rows` of every stored matrix (Q_0 first, materialised
    when diagonal), quantised by the oracle entry by entry."""
    Qd = data.Q
    idx = torch.as_tensor(rows, device=Qd.device)
    raw = Qd.index_select(1, idx).cpu().numpy()                       # (M, k, n) float32
    out = []
    for i in range(raw.shape[0]):
        if storage == 0:
            out.append(raw[i].astype(np.float64))
        elif storage == 1:
            out.append(QZ.bf16_round(raw[i]).astype(np.float64))
        else:
            r, sp = QZ.jacobi_factors(Qd[i].diagonal().cpu().numpy())
            codes = QZ.fp8_jacobi_codes(raw[i], r[rows][:, None], r[None, :])
            out.append(sp[rows].astype(np.float64)[:, None] * QZ.e4m3_decode_table()[codes]
                       * sp.astype(np.float64)[None, :])
    if data.q0_kind == W.Q0_DIAG:
        q0 = np.zeros((len(rows), data.n))
        q0[np.arange(len(rows)), rows] = data.q0diag.cpu().numpy()[rows]
        out = [q0] + out
    return out


def check_pass_rows(R, data, storage, seed):
    s = R.Solver(data, bench_params(R, storage=storage, rows_per_block=0))
    n = data.n
    g = torch.Generator(device=data.Q.device)
    g.manual_seed(seed)
    lb, ub = data.lb, data.ub
    x = (lb + (ub - lb) * torch.rand(n, generator=g, device=lb.device)).contiguous()
    v = (1e-2 * torch.randn(n, generator=g, device=lb.device)).contiguous()
    U, Wt, dots = s.coupling_pass(x, v)
    tile = s.tile()
    s.close()
    rows = sample_rows(n, seed)
    mats = stored_rows(data, storage, rows)
    x64, v64 = x.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    U, Wt, dots = U.cpu().numpy(), Wt.cpu().numpy(), dots.cpu().numpy()
    c = data.c.cpu().numpy().astype(np.float64)
    assert len(mats) == U.shape[0] == data.m + 1
    for i, Qr in enumerate(mats):
        su = np.abs(Qr) @ np.abs(x64) + 1e-30
        sw = np.abs(Qr) @ np.abs(v64) + 1e-30
        eu = np.abs(U[i, rows] - Qr @ x64) / su
        ew = np.abs(Wt[i, rows] - Qr @ v64) / sw
        assert eu.max() <= 2e-6 * np.sqrt(n), (i, eu.max(), tile)
        assert ew.max() <= 2e-6 * np.sqrt(n), (i, ew.max(), tile)
        # the dots are float64 sums of the kernel's own float32 products:
        # equal to any other float64 summation order within n eps64 sum|terms|
        for j, a, b in ((0, x64, U[i]), (1, v64, Wt[i]), (3, x64, c[i]), (4, v64, c[i])):
            t = a * b.astype(np.float64)
            assert abs(dots[i, j] - t.sum()) <= 2.3e-16 * n * np.abs(t).sum() + 1e-300, (i, j)
    return tile


def check_stored_columns(R, data, storage, cols):
    """Q~ e_k is column k of the stored matrix: with one non-zero term per row
    the float32 result is the quantiser's value exactly (FP8: the two scale
    products in the kernel's order)."""
    s = R.Solver(data, bench_params(R, storage=storage, rows_per_block=0))
    dev = data.Q.device
    off = 1 if data.q0_kind == W.Q0_DIAG else 0
    for k in cols:
        e = torch.zeros(data.n, dtype=torch.float32, device=dev)
        e[k] = 1.0
        U, _, _ = s.coupling_pass(e, torch.zeros_like(e))
        U = U.cpu().numpy()
        for i in range(data.Q.shape[0]):
            col = data.Q[i, :, k].cpu().numpy()
            if storage == 1:
                ref = QZ.bf16_round(col)
            else:
                r, sp = QZ.jacobi_factors(data.Q[i].diagonal().cpu().numpy())
                dec = QZ.e4m3_decode_table()[QZ.fp8_jacobi_codes(col, r, r[k])].astype(np.float32)
                xs = np.float32(sp[k]) * np.float32(1.0)
                ref = ((dec * xs).astype(np.float32) * sp).astype(np.float32)
            np.testing.assert_array_equal(U[i + off], ref)
    s.close()


def oracle_problem(data):
    return O.Problem.from_data(data.numpy())


# ---------------------------------------------------------------------------
# Dense random QCQP, n = 4096, m = 50, float32 (the benchmark's workload)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def c2(cuda):
    d = W.config("C2", device=cuda)
    yield d
    del d
    torch.cuda.empty_cache()


def test_dense_4096x50_pass_sampled_rows(R, c2):
    tile = check_pass_rows(R, c2, 0, seed=11)
    assert tile["ctas"] > 0


def test_dense_4096x50_solve_meets_tolerance_in_the_oracle_kkt(R, cuda, c2):
    s = R.Solver(c2, bench_params(R))
    x = torch.zeros(c2.n, device=cuda)
    y = torch.zeros(c2.m, device=cuda)
    info = s.solve(x, y)
    x64, y64 = s.solution_f64()
    rel_gpu, _, _ = s.kkt_residual(x, y)
    s.close()
    assert info["status"] == R.OK and info["rel_kkt"] <= 1e-6, info
    prob = oracle_problem(c2)
    x64, y64 = x64.cpu().numpy(), y64.cpu().numpy()
    assert np.all(x64 >= prob.lb) and np.all(x64 <= prob.ub) and np.all(y64 >= 0)
    rel, _, _ = O.kkt_residual(prob, x64, y64)
    assert rel <= 1e-6, rel
    # the stand-alone residual (compensated products) at the float32 output
    rel32, _, _ = O.kkt_residual(prob, x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64))
    assert abs(rel_gpu - rel32) <= 1e-3 * rel32, (rel_gpu, rel32)
    assert abs(info["obj"] - prob.f(x64)) <= 1e-6 * (1 + abs(prob.f(x64)))


@pytest.mark.parametrize("variant,storage", [(0, 1), (0, 2), (1, 0)])
def test_dense_4096x50_other_forms_meet_tolerance(R, cuda, c2, variant, storage):
    """BF16 and FP8 storage with refinement (yx), and the xy variant with
    float32 storage, on the full workload: each ends at rel KKT 1e-6 by its
    own test, confirmed by the oracle's float64 residual at its iterate."""
    s = R.Solver(c2, bench_params(R, storage=storage, variant=variant))
    x = torch.zeros(c2.n, device=cuda)
    y = torch.zeros(c2.m, device=cuda)
    info = s.solve(x, y)
    x64, y64 = s.solution_f64()
    s.close()
    assert info["status"] == R.OK and info["rel_kkt"] <= 1e-6, info
    if storage != 0:
        assert info["precision_switches"] == 1, info
    prob = oracle_problem(c2)
    rel, _, _ = O.kkt_residual(prob, x64.cpu().numpy(), y64.cpu().numpy())
    assert rel <= 1e-6, rel


# ---------------------------------------------------------------------------
# Kernel-learning epigraph QCQP, n = 5000 samples, m = 8 kernels, bfloat16
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def c3(cuda):
    d = W.config("C3", device=cuda)
    yield d
    del d
    torch.cuda.empty_cache()


def test_kml_5001x8_bf16_pass_sampled_rows(R, c3):
    check_pass_rows(R, c3, 1, seed=12)


def test_kml_5001x8_bf16_stored_columns_bit_exact(R, c3):
    check_stored_columns(R, c3, 1, cols=(0, 2500, 4999, 5000))


def test_kml_5001x8_bf16_iterates_stay_feasible_and_kkt_agrees(R, cuda, c3):
    """A bounded run (the epigraph form converges slowly for this method;
    the oracle behaves the same): box and sign feasibility of the result,
    and the library's stand-alone KKT residual equals the oracle's."""
    s = R.Solver(c3, bench_params(R, storage=1, max_iter=600))
    x = torch.zeros(c3.n, device=cuda)
    y = torch.zeros(c3.m, device=cuda)
    info = s.solve(x, y, check=False)
    assert info["status"] in (R.OK, R.ERR_MAXITER), info
    rel_gpu, rs_gpu, rf_gpu = s.kkt_residual(x, y)
    s.close()
    prob = oracle_problem(c3)
    xh, yh = x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64)
    assert np.all(xh >= prob.lb) and np.all(xh <= prob.ub) and np.all(yh >= 0)
    rel, rs, rf = O.kkt_residual(prob, xh, yh)
    assert abs(rel_gpu - rel) <= 1e-3 * rel, (rel_gpu, rel)
    assert abs(rs_gpu - rs) <= 1e-3 * rs and abs(rf_gpu - rf) <= 1e-3 * rf + 1e-12


# ---------------------------------------------------------------------------
# 256 random QCQPs of uneven sizes in one batched device loop
# ---------------------------------------------------------------------------

def test_batched_256_sampled_instances(R, cuda):
    datas = W.batched_random_qcqp(256, seed=0)
    devs = [d.to(cuda) for d in datas]
    p = R.Params.default(R.YX, tol=1e-6, max_iter=20000, time_limit_s=120.0, refine=1)
    bs = R.BatchedSolver(devs, p)
    xs = [torch.zeros(d.n, device=cuda) for d in datas]
    ys = [torch.zeros(max(d.m, 1), device=cuda) for d in datas]
    infos = bs.solve(xs, ys)
    tiles = [bs.tile(b) for b in range(len(datas))]
    bs.close()
    assert all(i["status"] == R.OK and i["rel_kkt"] <= 1e-6 for i in infos)
    order = np.argsort([d.n for d in datas])
    # the two smallest instances: the oracle's own solve reaches the same objective
    for b in order[:2]:
        prob = O.Problem.from_data(datas[b])
        r = O.rapdb(prob, p=O.default_params("yx", tol=1e-6, restart_period=200))
        xb = xs[b].cpu().numpy().astype(np.float64)
        fo, fg = prob.f(r.x), prob.f(xb)
        assert abs(fg - fo) <= 1e-5 * (1 + abs(fo)), (b, fg, fo)
    # the batched loop drops finished instances from its launch grids as they
    # finish; each instance's arithmetic is unchanged, so a single-instance
    # context with the instance's (autotuned) tile ends on the same bits; its
    # float64 iterate then gives the oracle's float64 KKT residual at the
    # solver's own point, held to the tolerance 1e-6 (the float32 copy the
    # batched call returns adds its rounding, about 1e-7 relative, on top)
    for b in list(order[::64]) + [order[len(order) // 2], order[-1]]:
        ps = R.Params.default(R.YX, tol=1e-6, max_iter=20000, time_limit_s=120.0, refine=1,
                              rows_per_block=tiles[b]["rows_per_block"], pass_variant=tiles[b]["variant"])
        s1 = R.Solver(devs[b], ps)
        x1 = torch.zeros(datas[b].n, device=cuda)
        y1 = torch.zeros(max(datas[b].m, 1), device=cuda)
        i1 = s1.solve(x1, y1)
        x64, y64 = s1.solution_f64()
        s1.close()
        assert i1["iters"] == infos[b]["iters"], (b, i1["iters"], infos[b]["iters"])
        assert torch.equal(x1, xs[b]) and torch.equal(y1, ys[b]), b
        prob = O.Problem.from_data(datas[b])
        xg, yg = x64.cpu().numpy(), y64.cpu().numpy()[: datas[b].m]
        assert np.all(xg >= prob.lb) and np.all(xg <= prob.ub) and np.all(yg >= 0)
        rel, _, _ = O.kkt_residual(prob, xg, yg)
        assert rel <= 1e-6, (b, datas[b].n, datas[b].m, rel)
        xb = xs[b].cpu().numpy().astype(np.float64)
        yb = ys[b].cpu().numpy().astype(np.float64)[: datas[b].m]
        rel32, _, _ = O.kkt_residual(prob, xb, yb)
        assert rel32 <= 1e-5, (b, rel32)
    del devs
    torch.cuda.empty_cache()


# ---------------------------------------------------------------------------
# Kernel-learning epigraph QCQP, n = 16000 samples, m = 20 kernels, FP8
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def c5(cuda):
    d = W.config("C5", device=cuda)
    yield d
    del d
    torch.cuda.empty_cache()


def test_kml_16001x20_fp8_pass_sampled_rows(R, c5):
    check_pass_rows(R, c5, 2, seed=13)


def test_kml_16001x20_fp8_stored_columns_bit_exact(R, c5):
    check_stored_columns(R, c5, 2, cols=(0, 16000))
