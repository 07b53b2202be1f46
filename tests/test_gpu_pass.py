"""The fused coupling pass (the hot operator) against float64 products with the
stored matrices: float32, bfloat16 and Jacobi-scaled FP8 storage, dense,
diagonal and zero Q_0, ragged sizes that leave partial row blocks and partial
16-byte column vectors."""
import numpy as np
import pytest
import torch

from oracle import quant as QZ
from paper_2605_29291_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def stored_q(data, storage):
    """float64 matrices the library stores (the oracle's quantisers)."""
    h = data.numpy()
    out = []
    for Qi in h.Q:
        if storage == 0:
            out.append(Qi.astype(np.float64))
        elif storage == 1:
            out.append(QZ.bf16_round(Qi).astype(np.float64))
        else:
            codes, s = QZ.fp8_jacobi_quantize(Qi)
            out.append(QZ.fp8_dequantize(codes, s))
    return out


def make(n, m, q0_kind, seed):
    rng = np.random.default_rng(seed)
    if q0_kind == W.Q0_DENSE:
        return W.random_qcqp(n, m, rows=max(n // 2, 1), seed=seed)
    base = W.random_qcqp(n, m, rows=max(n // 2, 1), seed=seed)
    q0diag = rng.uniform(0.5, 2.0, n).astype(np.float32) if q0_kind == W.Q0_DIAG else None
    return W.QCQPData(n, m, base.Q[1:].copy(), base.c, base.d, base.lb, base.ub, q0_kind, q0diag)


CASES = [(200, 10, W.Q0_DENSE), (203, 3, W.Q0_DENSE), (67, 1, W.Q0_DENSE), (1000, 2, W.Q0_DENSE),
         (131, 4, W.Q0_DIAG), (96, 2, W.Q0_ZERO), (50, 0, W.Q0_DENSE), (9, 2, W.Q0_DENSE)]


@pytest.mark.parametrize("storage", [0, 1, 2])
@pytest.mark.parametrize("n,m,q0_kind", CASES)
def test_pass_matches_float64(R, cuda, storage, n, m, q0_kind):
    data = make(n, m, q0_kind, seed=n + 7 * m)
    dev = data.to(cuda)
    s = R.Solver(dev, R.Params.default(storage=storage))
    rng = np.random.default_rng(1)
    x = rng.uniform(-3, 3, n).astype(np.float32)
    v = rng.standard_normal(n).astype(np.float32) * 1e-3
    uold = rng.standard_normal((m + 1, n)).astype(np.float32)
    U, Wt, dots = s.coupling_pass(torch.from_numpy(x).to(cuda), torch.from_numpy(v).to(cuda),
                                  torch.from_numpy(uold).to(cuda))
    U, Wt, dots = U.cpu().numpy(), Wt.cpu().numpy(), dots.cpu().numpy()
    Qs = stored_q(data, storage)
    h = data.numpy()
    mats = list(Qs)
    if q0_kind == W.Q0_DIAG:
        mats = [np.diag(h.q0diag.astype(np.float64))] + mats
    elif q0_kind == W.Q0_ZERO:
        mats = [np.zeros((n, n))] + mats
    x64, v64 = x.astype(np.float64), v.astype(np.float64)
    for i, Qi in enumerate(mats):
        ref_u, ref_w = Qi @ x64, Qi @ v64
        scale_u = np.abs(Qi) @ np.abs(x64) + 1e-30
        scale_w = np.abs(Qi) @ np.abs(v64) + 1e-30
        # float32 accumulation over n terms: relative to sum |Q_jk x_k|
        assert np.all(np.abs(U[i] - ref_u) <= 2e-6 * np.sqrt(n) * scale_u + 1e-37), (i, np.max(np.abs(U[i] - ref_u) / scale_u))
        assert np.all(np.abs(Wt[i] - ref_w) <= 2e-6 * np.sqrt(n) * scale_w + 1e-37)
        ci = h.c[i].astype(np.float64)
        # the dots are float64 sums of the kernel's own float32 products
        np.testing.assert_allclose(dots[i, 0], x64 @ U[i].astype(np.float64), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(dots[i, 1], v64 @ Wt[i].astype(np.float64), rtol=1e-12, atol=1e-18)
        np.testing.assert_allclose(dots[i, 2], v64 @ uold[i].astype(np.float64), rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(dots[i, 3], ci @ x64, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(dots[i, 4], ci @ v64, rtol=1e-12, atol=1e-15)
    s.close()


@pytest.mark.parametrize("storage", [1, 2])
def test_stored_codes_bit_exact(R, cuda, storage):
    """Q e_k returns column k of the stored matrix; with one non-zero term per
    row the float32 result is exactly the quantiser's value (FP8: the two
    scale products in the kernel's order)."""
    n, m = 72, 2
    data = W.random_qcqp(n, m, rows=30, seed=3)
    s = R.Solver(data.to(cuda), R.Params.default(storage=storage))
    h = data.numpy()
    for k in (0, 5, 71):
        e = torch.zeros(n, dtype=torch.float32, device=cuda)
        e[k] = 1.0
        U, _, _ = s.coupling_pass(e, torch.zeros_like(e))
        U = U.cpu().numpy()
        for i in range(m + 1):
            if storage == 1:
                ref = QZ.bf16_round(h.Q[i][:, k].copy())
            else:
                codes, sc = QZ.fp8_jacobi_quantize(h.Q[i])
                dec = QZ.e4m3_decode_table()[codes[:, k]].astype(np.float32)
                xs = np.float32(sc[k]) * np.float32(1.0)
                ref = ((dec * xs).astype(np.float32) * sc).astype(np.float32)
            np.testing.assert_array_equal(U[i], ref)   # values: +0 and -0 compare equal
    s.close()


def test_pass_is_deterministic(R, cuda):
    data = W.random_qcqp(500, 6, rows=200, seed=9)
    s = R.Solver(data.to(cuda))
    x = torch.randn(500, device=cuda)
    v = torch.randn(500, device=cuda)
    a = s.coupling_pass(x, v)
    b = s.coupling_pass(x, v)
    for p, q in zip(a, b):
        assert torch.equal(p, q)
    s.close()


@pytest.mark.parametrize("variant", range(10))
@pytest.mark.parametrize("storage", [0, 1, 2])
@pytest.mark.parametrize("n,m,q0_kind", [(203, 3, W.Q0_DENSE), (1000, 2, W.Q0_DIAG), (37, 1, W.Q0_DENSE)])
def test_every_tile_variant(R, cuda, variant, storage, n, m, q0_kind):
    """Each coupling-pass tile the autotuner can pick (register streaming,
    per-warp bulk-copy slots, whole-row bulk-copy stages) gives the same
    products as float64 with the stored matrices."""
    data = make(n, m, q0_kind, seed=3 * n + m)
    s = R.Solver(data.to(cuda), R.Params.default(storage=storage, rows_per_block=32, pass_variant=variant))
    assert s.tile()["rows_per_block"] == 32
    rng = np.random.default_rng(2)
    x = rng.uniform(-3, 3, n).astype(np.float32)
    v = rng.standard_normal(n).astype(np.float32)
    U, Wt, dots = s.coupling_pass(torch.from_numpy(x).to(cuda), torch.from_numpy(v).to(cuda))
    U, Wt, dots = U.cpu().numpy(), Wt.cpu().numpy(), dots.cpu().numpy()
    h = data.numpy()
    mats = stored_q(data, storage)
    if q0_kind == W.Q0_DIAG:
        mats = [np.diag(h.q0diag.astype(np.float64))] + mats
    x64, v64 = x.astype(np.float64), v.astype(np.float64)
    for i, Qi in enumerate(mats):
        scale_u = np.abs(Qi) @ np.abs(x64) + 1e-30
        scale_w = np.abs(Qi) @ np.abs(v64) + 1e-30
        assert np.all(np.abs(U[i] - Qi @ x64) <= 2e-6 * np.sqrt(n) * scale_u)
        assert np.all(np.abs(Wt[i] - Qi @ v64) <= 2e-6 * np.sqrt(n) * scale_w)
        np.testing.assert_allclose(dots[i, 0], x64 @ U[i].astype(np.float64), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(dots[i, 1], v64 @ Wt[i].astype(np.float64), rtol=1e-12, atol=1e-12)
    s.close()


@pytest.mark.parametrize("variant", range(10))
def test_every_tile_variant_solves(R, cuda, variant):
    """The full device loop with each tile variant reaches the oracle's
    objective on a ragged instance."""
    import oracle as O
    data = W.random_qcqp(203, 3, seed=203)
    s = R.Solver(data.to(cuda), R.Params.default(tol=1e-6, max_iter=20000, rows_per_block=64,
                                                 pass_variant=variant))
    x = torch.zeros(203, device=cuda)
    y = torch.zeros(3, device=cuda)
    info = s.solve(x, y)
    assert info["status"] == R.OK
    prob = O.Problem.from_data(data)
    r = O.rapdb(prob, p=O.default_params("yx", tol=1e-6, max_iter=20000))
    fo = prob.f(r.x)
    assert abs(info["obj"] - fo) <= 1e-5 * (1 + abs(fo))
    s.close()
