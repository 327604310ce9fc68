"""The paper's own synthetic workloads (Section 5): circular ring and cube.

CPU: the generators follow the stated construction -- the ring is one loop of
radius 2 with m = n; the cube's mean edge count matches the paper's
E(m) = 2 (2 n^3 - 3 n^2 + 1) p + n^3 - 1 and every edge joins grid neighbours.
GPU: the library matches the oracle on them (FP64 1e-10, FP32 1e-5 per array
after 1 and 10 iterations; per element, FP64 within 1e-10 of each element's
scale and FP32 by the FP32 rule of tests/parity.py against the oracle's
single-precision execution and its FP32-storage run) and, with the paper's
settings (tau = 1.4, tol = 1e-4, MaxIter = 300), its FP64 solve stops at the
oracle's iteration.
"""
import numpy as np
import pytest

import oracle
from paper_2601_15684_gb300 import synth
from parity import ELEM_TOL_FP64, check_elements, check_elements_fp32, fp32_storage_run

WORKLOADS = ("ring100", "ring5000", "cube7", "cube10")


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_ring_construction():
    g = synth.ring_graph(100)
    assert g.n == 100 and g.m == 100
    np.testing.assert_allclose(np.linalg.norm(g.t_gt[:, :2], axis=1), 2.0, rtol=1e-15)
    assert (g.dst == (g.src + 1) % 100).all()
    # orientation tangent to the loop: the heading (body x axis) is the direction of travel
    x_body = synth._rotate(g.q_gt, np.tile([1.0, 0.0, 0.0], (g.n, 1)))
    step = np.roll(g.t_gt, -1, axis=0) - g.t_gt
    cos = (x_body * step).sum(1) / np.linalg.norm(step, axis=1)
    assert cos.min() > 0.99


@pytest.mark.parametrize("side,p", [(2, 0.3), (7, 0.3), (10, 0.9)])
def test_cube_construction(side, p):
    ms = []
    for seed in range(24):
        g = synth.cube_graph(side, p, seed=seed)
        d = np.linalg.norm(g.t_gt[g.dst] - g.t_gt[g.src], axis=1)
        np.testing.assert_allclose(d, 2.0 / (side - 1), rtol=1e-12)  # grid neighbours only
        assert g.n == side ** 3 and (g.src != g.dst).all()
        ms.append(g.m)
    expected = 2 * (2 * side ** 3 - 3 * side ** 2 + 1) * p + side ** 3 - 1
    # closures are 2 (2 n^3 - 3 n^2 + 1) Bernoulli(p) draws: mean within 4 standard errors
    sd = np.sqrt(2 * (2 * side ** 3 - 3 * side ** 2 + 1) * p * (1 - p) / len(ms))
    assert abs(np.mean(ms) - expected) <= 4 * sd + 1e-9


def test_oracle_solves_paper_workloads_noise_free():
    # noise-free ring / cube started at the truth is a fixed point of the oracle
    for g in (synth.ring_graph(100, sigma_r=0.0, sigma_t=0.0), synth.cube_graph(4, 0.5, sigma_r=0.0, sigma_t=0.0)):
        st = oracle.init_state(g.q_gt, g.t_gt)
        x, res, _ = oracle.iterate(g, oracle.make_params(beta1=1.0, beta2=1.0, tau=1.4), st, 1)
        assert res[0] < 1e-24
        assert relerr(x["t"], g.t_gt) < 1e-13


@pytest.fixture(scope="module")
def P():
    from paper_2601_15684_gb300 import build_lib
    from paper_2601_15684_gb300 import pradmm
    build_lib.build()
    pradmm.load()
    return pradmm


def _prm(P, precision, tau=1.4):
    prm = P.pradmm_default_params()
    prm.relax = tau
    prm.precision = precision
    prm.tol = 1e-4
    prm.max_iter = 300
    return prm


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", WORKLOADS)
def test_paper_workloads_match_oracle(P, name, precision):
    g = synth.workload(name)
    op = oracle.make_params(beta1=1.0, beta2=1.0, tau=1.4)
    q0, t0 = oracle.init_odometry(g)
    orc = oracle.init_state(q0, t0)
    orc32, orcx = orc, orc
    step = lambda st: oracle.iterate(g, op, st, 1)[0]
    with P.Solver(g, _prm(P, precision)) as S:
        S.init_odometry()
        done = 0
        for it in (1, 10):
            S.step(it - done)
            orc, _, _ = oracle.iterate(g, op, orc, it - done)
            if precision == 1:
                orc32 = fp32_storage_run(step, orc32, it - done)
                orcx = oracle.iterate_f32(g, op, orcx, it - done)
            done = it
            gpu = S.state()
            tol = 1e-10 if precision == 0 else 1e-5
            for key in ("p", "q", "t", "s"):
                assert relerr(gpu[key], orc[key]) <= tol, (name, it, key, relerr(gpu[key], orc[key]))
            what = f"{name} after {it}"
            if precision == 0:
                check_elements(gpu, orc, ELEM_TOL_FP64, what=what, tau=1.4)
            else:
                check_elements_fp32(gpu, orc, [orc32, orcx], what=what, tau=1.4)


@pytest.mark.gpu
@pytest.mark.parametrize("name", WORKLOADS)
def test_paper_settings_solve_stops_like_oracle(P, name):
    g = synth.workload(name)
    q0, t0 = oracle.init_odometry(g)
    st, k, e, _ = oracle.solve(g, oracle.make_params(beta1=1.0, beta2=1.0, tau=1.4), oracle.init_state(q0, t0),
                               300, 1e-4)
    with P.Solver(g, _prm(P, 0)) as S:
        S.init_odometry()
        converged, iters, e_gpu = S.solve()
        F = S.objective()
    assert iters == k and converged == (e < 1e-4)
    F_ref = oracle.objective(g, st["p"], st["t"])
    assert abs(F - F_ref) <= 1e-6 * max(F_ref, 1e-12)
