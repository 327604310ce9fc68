"""Small driver for profiling the sweep kernels under Nsight Compute.

Builds one named synthetic workload, initialises it by odometry and runs a
few PRADMM iterations with plain stream launches (one kernel per launch,
so `ncu -k regex:... -s ... -c ...` can pick single sweeps), then exits.

    python -m paper_2601_15684_gb300.prof_run --workload lattice1m --iters 12
"""
from __future__ import annotations

import argparse
import sys
import time


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="lattice1m")
    ap.add_argument("--iters", type=int, default=12)
    ap.add_argument("--precision", type=int, default=1)
    ap.add_argument("--graph", type=int, default=0)
    ap.add_argument("--block", type=int, default=0)
    a = ap.parse_args(argv)
    from paper_2601_15684_gb300 import build_lib, pradmm, synth

    build_lib.build()
    g = synth.workload(a.workload)
    with pradmm.Solver(g, precision=a.precision, use_graph=a.graph, block=a.block) as S:
        S.init_odometry()
        t0 = time.perf_counter()
        e = S.step(a.iters)
        dt = time.perf_counter() - t0
        print(f"{a.workload}: n={g.n} m={g.m} iters={a.iters} e={e:.6e} wall={dt * 1e3:.2f} ms "
              f"bytes/iter={S.bytes_per_iteration()['total']:.4e}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
