"""Failure detection without a GPU fault: the bounded mbarrier wait that
guards every bulk-copy stage of the coupling pass gives up at its limit, sets
the error flag and returns, and the device stays usable afterwards."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_wait_returns_when_the_copy_completes(R):
    r = R.wait_selftest(True, limit_us=50000)
    assert not r["gave_up"]
    assert r["copied_sum"] == 10.0
    assert r["waited_ms"] < 50.0


@pytest.mark.parametrize("limit_us", [2000, 20000])
def test_wait_gives_up_at_its_limit_and_the_device_stays_usable(R, limit_us):
    r = R.wait_selftest(False, limit_us=limit_us)
    assert r["gave_up"]
    assert r["copied_sum"] == -1.0
    assert limit_us / 1000.0 <= r["waited_ms"] < limit_us / 1000.0 + 500.0
    # the context is intact: a solve on the same device runs to optimality
    from paper_2605_29291_gb300 import workloads as W
    data = W.random_qcqp(64, 3, rows=32, seed=5, device="cuda:0")
    s = R.Solver(data, R.Params.default(R.YX, tol=1e-5, rows_per_block=32, pass_variant=2))
    info = s.solve(torch.zeros(64, device="cuda:0"), torch.zeros(3, device="cuda:0"))
    s.close()
    assert info["status"] == R.OK and info["rel_kkt"] <= 1e-5
    torch.cuda.synchronize()
