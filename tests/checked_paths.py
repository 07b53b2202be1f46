"""Runs every solver path once under the checked build of the library (the
kernels verify their block indices and launch shapes and report a failed
check as an error status).  Started by tests/test_gpu_checked.py with
RAPDB_LIBRARY pointing at librapdb_checked.so; prints 'checked paths ok'."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2605_29291_gb300 import rapdb as R  # noqa: E402
from paper_2605_29291_gb300 import workloads as W  # noqa: E402

assert os.path.basename(R.LIB_PATH) == "librapdb_checked.so", R.LIB_PATH
dev = torch.device("cuda:0")


def run(data, params, y0=None):
    s = R.Solver(data.to(dev), params)
    x = torch.zeros(data.n, device=dev)
    y = torch.zeros(max(s.m, 1), device=dev) if y0 is None else y0
    info = s.solve(x, y)
    assert info["status"] in (R.OK, R.ERR_MAXITER), info
    s.kkt_residual(x, y)
    s.coupling_pass(torch.rand(data.n, device=dev), torch.rand(data.n, device=dev))
    if params.pack_sym:
        M = int(data.Q.shape[0])
        s.packed_pass(torch.rand(data.n, device=dev), torch.rand(data.n, device=dev),
                      torch.rand((M, data.n), device=dev))
    for level in (0, 1, 2, 3, 4, 5):
        try:
            s.time_pass(reps=1, level=level)
        except R.RapdbError as e:
            if e.status != R.ERR_INVALID:         # a level the context does not have
                raise
    s.close()


dense = W.random_qcqp(203, 3, rows=101, seed=1)
base = W.random_qcqp(131, 4, rows=65, seed=2)
diag = W.QCQPData(131, 4, base.Q[1:].copy(), base.c, base.d, base.lb, base.ub, W.Q0_DIAG,
                  np.random.default_rng(0).uniform(0.5, 2.0, 131).astype(np.float32))
for storage in (0, 1, 2):
    for rb, var in ((0, 0), (32, 0), (64, 1), (64, 2), (64, 3), (128, 4), (64, 5), (64, 6), (128, 8), (64, 9)):
        for data in (dense, diag):
            run(data, R.Params.default(R.YX, storage=storage, refine=1, rows_per_block=rb, pass_variant=var,
                                       tol=1e-5, max_iter=2000))
# xy, adaptive restart, average restart
run(dense, R.Params.default(R.XY, tol=1e-5, max_iter=3000, restart=R.RESTART_GAP, gap_first=50, gap_every=100))
run(dense, R.Params.default(R.YX, tol=1e-5, max_iter=3000, restart_from_average=1, restart_period=100))
# simplex dual with an equality
kb = W.kml_minmax(150, 5, 3, seed=1, bias=True)
y0 = torch.tensor([1 / 3, 1 / 3, 1 / 3, 0.0], device=dev)
run(kb, R.Params.default(R.YX, dual_set=R.DUAL_SIMPLEX, tol=1e-5, max_iter=3000), y0)
# symmetric block packing: float32, BF16 and FP8 storage, dense and diagonal Q_0, yx and xy
for storage in (0, 1, 2):
    for data in (dense, diag):
        run(data, R.Params.default(R.YX, storage=storage, refine=1, pack_sym=1, tol=1e-5, max_iter=2000))
run(dense, R.Params.default(R.XY, pack_sym=1, tol=1e-5, max_iter=3000, restart=R.RESTART_GAP, gap_first=50,
                            gap_every=100))
run(kb, R.Params.default(R.YX, dual_set=R.DUAL_SIMPLEX, pack_sym=1, tol=1e-5, max_iter=3000), y0)
# batched, with finished instances dropped from the grids as they finish
datas = W.batched_random_qcqp(48, seed=5, n_lo=32, n_hi=300, m_lo=1, m_hi=8)
bs = R.BatchedSolver([d.to(dev) for d in datas], R.Params.default(tol=1e-6, max_iter=20000))
xs = [torch.zeros(d.n, device=dev) for d in datas]
ys = [torch.zeros(max(d.m, 1), device=dev) for d in datas]
infos = bs.solve(xs, ys)
assert all(i["status"] == R.OK for i in infos)
infos = bs.solve(xs, ys)      # a second solve on the restored full maps
assert all(i["status"] == R.OK for i in infos)
bs.close()
torch.cuda.synchronize()
print("checked paths ok")
