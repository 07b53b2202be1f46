"""Time the fused coupling pass on a synthetic random QCQP of a chosen size.

    python -m paper_2605_29291_gb300.passbench --n 4096 --m 10 [--storage 0|1|2]
        [--rows-per-block 0|32|64|...] [--variant 0..9] [--reps 3] [--level -1..7]
        [--pack]

The instance is ``workloads.random_qcqp(n, m, rows=n/2)`` built on the GPU.
With ``--rows-per-block 0`` the library's autotuner picks the tile; otherwise
the given rows per CTA and tile variant are used; ``--pack`` builds the
symmetric block packing (level 4 times the packed incremental pass, level 5
its tile kernel alone; with ``--storage 1|2`` levels 6 and 7 time the same
over the packed BF16 / FP8 tiles; see rapdb_time_pass).  The
pass is launched once
to warm up, then ``--reps`` times between two CUDA events on the context's
stream; the line printed gives the tile, the time per launch and the
algorithmic bytes per second.  The launch sequence is fixed, so the command
also serves as a profiling target (one warm-up launch, then the timed ones).
"""
from __future__ import annotations

import argparse


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--m", type=int, default=10)
    ap.add_argument("--storage", type=int, default=0)
    ap.add_argument("--rows-per-block", type=int, default=0)
    ap.add_argument("--variant", type=int, default=0)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--level", type=int, default=0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--pack", action="store_true")
    a = ap.parse_args(argv)
    import torch

    from . import rapdb as R
    from . import workloads as W
    dev = torch.device("cuda:0")
    data = W.random_qcqp(a.n, a.m, rows=max(a.n // 2, 1), seed=a.seed, device=dev)
    s = R.Solver(data, R.Params.default(storage=a.storage, rows_per_block=a.rows_per_block,
                                        pass_variant=a.variant, refine=1, pack_sym=int(a.pack)))
    ms, b = s.time_pass(reps=a.reps, level=a.level)
    print(f"tile {s.tile()} level {a.level}: {ms * 1e3:.1f} us per pass, {b / 1e6:.1f} MB, "
          f"{b / (ms * 1e-3) / 1e9:.0f} GB/s")
    s.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
