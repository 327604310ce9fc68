"""The OpenMP timing build of the oracle (the benchmark's multi-core CPU
baseline) against the single-threaded checker: the same iteration with every
block's loop over vertices, each vertex summing its own edges in input order,
so the state is bitwise the checker's and the residual agrees to rounding."""
import os

import numpy as np
import pytest

import oracle
from paper_2601_15684_gb300 import synth


@pytest.mark.parametrize("case", ["ragged", "isolated", "walk128"])
def test_openmp_build_state_is_bitwise_the_checkers(case):
    if case == "ragged":
        g = synth.random_graph(3000, 9000, seed=1)
    elif case == "isolated":
        g = synth.random_graph(1200, 2500, seed=3, isolated=300)
    else:
        g = synth.workload("walk128")
    st0 = synth.random_state(np.random.default_rng(10), g.n)
    prm = oracle.make_params(beta1=3.0, beta2=5.0, tau=1.3, gamma=(0.7, 0.01, 0.02, 0.03))
    ref, res, _ = oracle.iterate(g, prm, st0, 5)
    got, trace = oracle.iterate_omp(g, prm, st0, 5)
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    assert abs(trace[-1] - res[0]) <= 1e-12 * res[0]


def test_openmp_build_uses_the_requested_threads():
    # the thread count reported with the baseline is the one the build runs on
    assert oracle.omp_threads() >= 1
    if os.environ.get("OMP_NUM_THREADS"):
        assert oracle.omp_threads() == int(os.environ["OMP_NUM_THREADS"])


def test_single_precision_build_is_fp32_and_close():
    # the tolerance reference: the checker's algorithm in FP32 arithmetic
    # stays within FP32 rounding of the FP64 oracle on a well-conditioned
    # walk, and it really rounds to FP32 (it is not the FP64 build)
    g = synth.workload("walk128")
    q0, t0 = oracle.init_odometry(g)
    st0 = oracle.init_state(q0, t0)
    prm = oracle.make_params(beta1=1.0, beta2=1.0, tau=1.5)
    ref, _, _ = oracle.iterate(g, prm, st0, 10)
    got = oracle.iterate_f32(g, prm, st0, 10)
    for k in ("p", "q", "t", "s"):
        e = np.linalg.norm(got[k] - ref[k]) / np.linalg.norm(ref[k])
        assert 1e-9 < e < 1e-5, (k, e)
        assert np.array_equal(got[k], got[k].astype(np.float32).astype(np.float64))
    pr, _, _, _ = oracle.iterate_inertial(g, prm, st0, 0.4, 6)
    pf, _ = oracle.iterate_inertial_f32(g, prm, st0, 0.4, 6)
    for k in ("p", "t"):
        e = np.linalg.norm(pf[k] - pr[k]) / np.linalg.norm(pr[k])
        assert 1e-9 < e < 1e-5, (k, e)
