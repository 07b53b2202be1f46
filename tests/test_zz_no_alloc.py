"""The allocation-free coupling pass (rapdb_coupling_pass_noalloc), called
through the C ABI, against the context-based rapdb_coupling_pass.

The allocation-free call serves callers that cannot allocate device memory:
code inside another framework's memory pool or a fixed memory budget,
real-time loops that must not enter the allocator, and code recording CUDA
graphs.  Its scratch is one fixed array shared by all calls on a device, so
the test makes two different calls in a row and checks both."""
import numpy as np
import pytest
import torch

from paper_2605_29291_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def reference_pass(R, cuda, data, x, v, uold):
    s = R.Solver(data.to(cuda), R.Params.default(rows_per_block=32, pass_variant=0))
    out = s.coupling_pass(x, v, uold)
    s.close()
    return out


def test_noalloc_matches_context_pass_twice(R, cuda):
    rng = np.random.default_rng(5)
    cases = [W.random_qcqp(200, 10, rows=100, seed=1), W.random_qcqp(1000, 3, rows=400, seed=2)]
    for data in cases:
        dev = data.to(cuda)
        n, M = data.n, data.m + 1
        x = torch.from_numpy(rng.uniform(-3, 3, n).astype(np.float32)).to(cuda)
        v = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).to(cuda)
        uold = torch.from_numpy(rng.standard_normal((M, n)).astype(np.float32)).to(cuda)
        U, Wt, dots = R.coupling_pass_noalloc(dev.Q, dev.c, x, v, uold)
        torch.cuda.synchronize()
        U0, W0, d0 = reference_pass(R, cuda, data, x, v, uold)
        Qs = data.numpy().Q.astype(np.float64)
        x64, v64 = x.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
        for i in range(M):
            scale_u = np.abs(Qs[i]) @ np.abs(x64) + 1e-30
            scale_w = np.abs(Qs[i]) @ np.abs(v64) + 1e-30
            # same tolerance as the pass parity tests, against the context pass
            assert np.all(np.abs(U[i].cpu().numpy() - U0[i].cpu().numpy()) <= 2e-6 * np.sqrt(n) * scale_u)
            assert np.all(np.abs(Wt[i].cpu().numpy() - W0[i].cpu().numpy()) <= 2e-6 * np.sqrt(n) * scale_w)
        np.testing.assert_allclose(dots.cpu().numpy(), d0.cpu().numpy(), rtol=1e-9, atol=1e-9)


def test_noalloc_rejects_sizes_beyond_its_scratch(R, cuda):
    # (m+1) * 5 * ceil(n/32) > 131072 partial sums: rejected before any launch
    n, m = 4096, 204
    Q = torch.zeros((1, 4, 4), device=cuda)   # never read: the size check comes first
    c = torch.zeros((m + 1, n), device=cuda)
    x = torch.zeros(n, device=cuda)
    with pytest.raises(R.RapdbError):
        R.lib.rapdb_coupling_pass_noalloc  # the symbol exists
        st = R.lib.rapdb_coupling_pass_noalloc(n, m, Q.data_ptr(), c.data_ptr(), x.data_ptr(), x.data_ptr(),
                                               None, c.data_ptr(), c.data_ptr(), c.data_ptr(), None)
        if st != R.OK:
            raise R.RapdbError(st, "rejected")
