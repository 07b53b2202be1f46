"""The checked build of the library (kernels verify their block indices,
row ranges and dynamic shared memory against the launch, and report a failed
check as an error status instead of touching memory) runs every solver path
clean: all storages and tile variants, dense and diagonal Q_0, xy, restarts,
the simplex dual with an equality, the symmetric block packing, and batched
solves whose launch grids shrink as instances finish."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_runs_every_path_clean(cuda):
    from paper_2605_29291_gb300 import build as B
    lib = B.build(checked=True)
    env = dict(os.environ, RAPDB_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_paths.py")], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-4000:])
    assert "checked paths ok" in r.stdout
