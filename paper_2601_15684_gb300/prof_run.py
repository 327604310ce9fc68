"""Small driver for profiling the sweep kernels under Nsight Compute.

Builds one named synthetic workload, initialises it by odometry and runs a
few PRADMM iterations with plain stream launches (one kernel per launch,
so `ncu -k regex:... -s ... -c ...` can pick single sweeps), then exits.

    python -m paper_2601_15684_gb300.prof_run --workload lattice1m --iters 12

With --adjoint K it records K iterations (checkpoint every --ckpt) and runs
the reverse sweeps once for a seeded cotangent.  With --sigma the iterations
use general weight matrices: Sigma_1 = Q diag(1, 2, 0.5, 4) Q^T (Q a seeded
random rotation) and Sigma_2 = diag(1, 0.5, 2, 1).  With --batch G it
instead solves G random-walk graphs of the batched workload's distribution
(log-uniform sizes in [50, 20000]) for exactly --iters iterations in one
persistent launch, with the schedule --schedule block,warp_max_n,cluster,
cluster_min_n (and the general weights above with --sigma).
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
    ap.add_argument("--adjoint", type=int, default=0)
    ap.add_argument("--ckpt", type=int, default=20, help="checkpoint spacing (0: chosen from free memory)")
    ap.add_argument("--sigma", action="store_true", help="general Sigma_1, Sigma_2")
    ap.add_argument("--inertia", type=float, default=0.0, help="theta of the inertial variant")
    ap.add_argument("--batch", type=int, default=0, help="number of graphs of a batched solve")
    ap.add_argument("--schedule", default="256,256,1,0", help="batched schedule: block,warp_max_n,cluster,cluster_min_n")
    a = ap.parse_args(argv)
    from paper_2601_15684_gb300 import build_lib, pradmm, synth

    build_lib.build()
    if a.batch > 0:
        graphs = synth.batch_graphs(count=a.batch)
        sch = [int(x) for x in a.schedule.split(",")]
        with pradmm.Batch(graphs, precision=a.precision, inertia=a.inertia) as B:
            if a.sigma:
                import numpy as np
                rng = np.random.default_rng(0)
                Q, _ = np.linalg.qr(rng.normal(size=(4, 4)))
                B.set_sigma(Q @ np.diag([1.0, 2.0, 0.5, 4.0]) @ Q.T, np.diag([1.0, 0.5, 2.0, 1.0]))
            B.set_schedule(*sch)
            B.init_odometry()
            t0 = time.perf_counter()
            B.solve(rel_tol=0.0, max_iter=a.iters)
            dt = time.perf_counter() - t0
            print(f"batch: graphs={a.batch} poses={B.N} iters={a.iters} schedule={tuple(sch)} "
                  f"wall={dt * 1e3:.2f} ms")
        return 0
    g = synth.workload(a.workload)
    with pradmm.Solver(g, precision=a.precision, use_graph=a.graph, block=a.block, inertia=a.inertia) as S:
        if a.sigma:
            import numpy as np
            rng = np.random.default_rng(0)
            Q, _ = np.linalg.qr(rng.normal(size=(4, 4)))
            S.set_sigma(Q @ np.diag([1.0, 2.0, 0.5, 4.0]) @ Q.T, np.diag([1.0, 0.5, 2.0, 1.0]))
        S.init_odometry()
        t0 = time.perf_counter()
        e = S.step(a.iters)
        dt = time.perf_counter() - t0
        print(f"{a.workload}: n={g.n} m={g.m} iters={a.iters} e={e:.6e} wall={dt * 1e3:.2f} ms "
              f"bytes/iter={S.bytes_per_iteration()['total']:.4e}")
        if a.adjoint > 0:
            import numpy as np
            rng = np.random.default_rng(0)
            S.adjoint_record(a.adjoint, a.ckpt)
            t0 = time.perf_counter()
            out = S.adjoint(rng.normal(size=(g.n, 4)), rng.normal(size=(g.n, 3)))
            dt = time.perf_counter() - t0
            print(f"adjoint: iters={a.adjoint} ckpt={a.ckpt} wall={dt * 1e3:.2f} ms "
                  f"|dL/dt_meas|={np.linalg.norm(out['t_meas']):.6e}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
