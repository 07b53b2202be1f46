"""The allocation-free coupling pass (rapdb_coupling_pass_noalloc), called
through the C ABI.

Some callers cannot allocate device memory: code running inside another
framework's memory pool or a fixed, pre-planned memory budget, real-time loops
that must not enter the allocator, and code recording CUDA graphs.  For them
the library offers this pass, whose only scratch is one fixed array shared by
every call on a device.  The test makes several different calls in a row
(so each call finds the previous call's partial sums in that array) and
checks every product against float64 products of the stored matrices, under
the bound the context pass is held to, and the dots against the context's
rapdb_coupling_pass.  It sits in its own file, collected last."""
import numpy as np
import pytest
import torch

from paper_2605_29291_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def context_pass(R, cuda, data, x, v, uold):
    s = R.Solver(data.to(cuda), R.Params.default(rows_per_block=32, pass_variant=0))
    out = s.coupling_pass(x, v, uold)
    s.close()
    return out


def check_against_float64(data, x, v, uold, U, Wt, dots):
    """Products within float32 accumulation error of float64 ones (the bound
    of the pass parity tests), dots the float64 sums of the products."""
    h = data.numpy()
    n, M = data.n, data.m + 1
    x64 = x.cpu().numpy().astype(np.float64)
    v64 = v.cpu().numpy().astype(np.float64)
    U, Wt, dots = U.cpu().numpy(), Wt.cpu().numpy(), dots.cpu().numpy()
    for i in range(M):
        Qi = h.Q[i].astype(np.float64)
        scale_u = np.abs(Qi) @ np.abs(x64) + 1e-30
        scale_w = np.abs(Qi) @ np.abs(v64) + 1e-30
        assert np.all(np.abs(U[i] - Qi @ x64) <= 2e-6 * np.sqrt(n) * scale_u + 1e-37)
        assert np.all(np.abs(Wt[i] - Qi @ v64) <= 2e-6 * np.sqrt(n) * scale_w + 1e-37)
        ci = h.c[i].astype(np.float64)
        np.testing.assert_allclose(dots[i, 0], x64 @ U[i].astype(np.float64), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(dots[i, 1], v64 @ Wt[i].astype(np.float64), rtol=1e-12, atol=1e-18)
        if uold is None:
            assert dots[i, 2] == 0.0
        else:
            u64 = uold[i].cpu().numpy().astype(np.float64)
            np.testing.assert_allclose(dots[i, 2], v64 @ u64, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(dots[i, 3], ci @ x64, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(dots[i, 4], ci @ v64, rtol=1e-12, atol=1e-15)


def test_noalloc_matches_float64_and_context_pass(R, cuda):
    rng = np.random.default_rng(5)
    cases = [(W.random_qcqp(200, 10, rows=100, seed=1), True), (W.random_qcqp(1000, 3, rows=400, seed=2), True),
             (W.random_qcqp(200, 10, rows=100, seed=3), False), (W.random_qcqp(132, 2, rows=60, seed=4), False)]
    for data, with_uold in cases:
        dev = data.to(cuda)
        n, M = data.n, data.m + 1
        x = torch.from_numpy(rng.uniform(-3, 3, n).astype(np.float32)).to(cuda)
        v = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).to(cuda)
        uold = torch.from_numpy(rng.standard_normal((M, n)).astype(np.float32)).to(cuda) if with_uold else None
        U, Wt, dots = R.coupling_pass_noalloc(dev.Q, dev.c, x, v, uold)
        torch.cuda.synchronize()
        check_against_float64(data, x, v, uold, U, Wt, dots)
        U0, W0, d0 = context_pass(R, cuda, data, x, v, uold)
        # the same kernel arithmetic as the context pass with the same tile
        np.testing.assert_allclose(dots.cpu().numpy(), d0.cpu().numpy(), rtol=1e-9, atol=1e-9)
        assert torch.equal(U.cpu(), U0.cpu()) and torch.equal(Wt.cpu(), W0.cpu())


def test_noalloc_rejects_sizes_beyond_its_scratch(R, cuda):
    # (m+1) * 5 * ceil(n/32) = 26215 * 5 > 131072 partial sums: rejected
    # before any launch.  Every buffer has the size the call would use, so a
    # broken check would still compute in bounds and fail only on the status.
    n, m = 4, 26214
    M = m + 1
    Q = torch.zeros((M, n, n), device=cuda)
    c = torch.zeros((M, n), device=cuda)
    x = torch.zeros(n, device=cuda)
    U = torch.zeros((M, n), device=cuda)
    Wt = torch.zeros((M, n), device=cuda)
    dots = torch.zeros((M, 5), dtype=torch.float64, device=cuda)
    st = R.lib.rapdb_coupling_pass_noalloc(n, m, Q.data_ptr(), c.data_ptr(), x.data_ptr(), x.data_ptr(), None,
                                           U.data_ptr(), Wt.data_ptr(), dots.data_ptr(), None)
    torch.cuda.synchronize()
    assert st == R.ERR_INVALID
    # one constraint fewer fits and runs
    st = R.lib.rapdb_coupling_pass_noalloc(n, m - 1, Q.data_ptr(), c.data_ptr(), x.data_ptr(), x.data_ptr(), None,
                                           U.data_ptr(), Wt.data_ptr(), dots.data_ptr(), None)
    torch.cuda.synchronize()
    assert st == R.OK
