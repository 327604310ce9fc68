"""General weight matrices on the GPU (pradmm_set_sigma) against the
general-Sigma oracle (itself pinned by brute force on S^3, the scalar
reduction and block minimality).

Tolerances, relerr per state array: FP64 1e-9 (the p-update's sphere-
constrained solve goes through an eigen-decomposition and a secular equation
on both sides, by different algorithms: Jacobi + Newton here, the
8x8 eigenproblem of Algorithm 2 in the oracle); FP32 1e-4 for p, q, t, s.
"""
import numpy as np
import pytest

import oracle
from oracle import general_sigma as gs
from paper_2601_15684_gb300 import synth
from parity import check_elements, check_elements_fp32, fp32_storage_run

pytestmark = pytest.mark.gpu
KEYS = ("p", "q", "t", "s", "lam", "z")
PARAMS = (1.0, 1.0, 1.5, (1.0, 1e-3, 1e-3, 1e-3))


@pytest.fixture(scope="module")
def P():
    from paper_2601_15684_gb300 import build_lib
    from paper_2601_15684_gb300 import pradmm
    build_lib.build()
    pradmm.load()
    return pradmm


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _spd(rng, cond=8.0):
    Q, _ = np.linalg.qr(rng.normal(size=(4, 4)))
    return Q @ np.diag(np.exp(rng.uniform(0, np.log(cond), 4))) @ Q.T


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-4)])
def test_general_sigma_matches_oracle(P, precision, tol):
    rng = np.random.default_rng(3)
    g = synth.random_graph(97, 300, seed=5, isolated=2)
    st = synth.random_state(rng, g.n)
    S1, S2 = _spd(rng), _spd(rng)
    orc = st
    orc32 = st
    step = lambda x: gs.iterate(g, PARAMS, S1, S2, x)[0]
    with P.Solver(g, precision=precision) as S:
        S.set_sigma(S1, S2)
        S.set_state_full(st)
        done = 0
        for it in (1, 10):
            S.step(it - done)
            for _ in range(it - done):
                orc, _, _ = gs.iterate(g, PARAMS, S1, S2, orc)
            orc32 = fp32_storage_run(step, orc32, it - done)
            done = it
            gpu = S.state()
            for key in ("p", "q", "t", "s"):
                assert relerr(gpu[key], orc[key]) <= tol, (it, key, relerr(gpu[key], orc[key]))
            if precision == 0:
                for key in ("lam", "z"):
                    assert relerr(gpu[key], orc[key]) <= tol, (it, key)
                check_elements(gpu, orc, tol, what=f"general Sigma after {it}")
            else:
                # the general path's FP32 rule: ten times the scalar path's floor,
                # as its per-array bound is ten times the scalar path's
                check_elements_fp32(gpu, orc, orc32, what=f"general Sigma after {it}", floor=1e-3)
        F = S.objective()
    assert abs(F - gs.objective(g, S1, S2, orc["p"], orc["t"])) <= (1e-10 if precision == 0 else 1e-4) * max(F, 1.0)


def test_identity_sigma_equals_scalar_path(P):
    g = synth.random_graph(120, 360, seed=8)
    st = synth.random_state(np.random.default_rng(2), g.n)
    out = []
    for use_sigma in (False, True):
        with P.Solver(g, precision=0) as S:
            if use_sigma:
                S.set_sigma(np.eye(4), np.eye(4))
            S.set_state_full(st)
            S.step(12)
            out.append(S.state())
    for key in KEYS:
        assert relerr(out[1][key], out[0][key]) <= 1e-12, key


def test_walk_with_anisotropic_weights_converges_like_oracle(P):
    rng = np.random.default_rng(1)
    g = synth.random_walk_graph(60, n_closures=40, sigma_r=0.02, sigma_t=0.1, seed=4)
    S1 = np.diag([1.0, 4.0, 1.0, 0.25])
    S2 = _spd(rng, 3.0)
    q0, t0 = oracle.init_odometry(g)
    orc = oracle.init_state(q0, t0)
    es = []
    for _ in range(60):
        orc, e, _ = gs.iterate(g, PARAMS, S1, S2, orc)
        es.append(e)
    with P.Solver(g, precision=0) as S:
        S.set_sigma(S1, S2)
        S.init_odometry()
        e_gpu = S.step(60)
        gpu = S.state()
    assert abs(e_gpu - es[-1]) <= 1e-7 * max(es[-1], 1e-30)
    assert es[-1] < 1e-2 * es[0]  # the residual falls (3e-3 of the first after 60 iterations)
    for key in KEYS:
        assert relerr(gpu[key], orc[key]) <= 1e-8, key
    check_elements(gpu, orc, 1e-8, what="anisotropic walk after 60")


def test_set_sigma_validation_and_reset(P):
    g = synth.random_graph(30, 80, seed=1)
    st = synth.random_state(np.random.default_rng(0), g.n)
    with P.Solver(g, precision=0) as S:
        bad = np.eye(4)
        bad[0, 1] = 0.5  # not symmetric
        for S1, S2 in ((bad, np.eye(4)), (np.eye(4), -np.eye(4)), (np.eye(4), None)):
            with pytest.raises(P.PRADMMError) as ei:
                S.set_sigma(S1, S2)
            assert ei.value.status == P.PRADMM_ERR_ARG
        nan = np.eye(4)
        nan[2, 2] = np.nan
        with pytest.raises(P.PRADMMError) as ei:
            S.set_sigma(nan, np.eye(4))
        assert ei.value.status == P.PRADMM_ERR_NONFINITE
        S.set_sigma(2.0 * np.eye(4), np.eye(4))
        S.set_state_full(st)
        with pytest.raises(P.PRADMMError) as ei:
            S.adjoint_record(3, 1)
        assert ei.value.status == P.PRADMM_ERR_STATE
        S.set_sigma(None, None)  # back to the scalar model
        S.set_state_full(st)
        S.step(5)
        a = S.state()
    ref, _, _ = oracle.iterate(g, oracle.make_params(beta1=1.0, beta2=1.0, tau=1.5), st, 5)
    for key in KEYS:
        assert relerr(a[key], ref[key]) <= 1e-10, key


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-5)])
def test_hard_case_of_the_p_update(P, precision, tol):
    # vertex 0's multiplier is chosen so that its b_1 has no component on the
    # bottom eigenvector of A_1 and |-(A_1 - a_min I)^+ b_1| < 1: the p-update
    # is the hard case of Lemma 1 on both sides (the FP32 handle re-solves it
    # in FP64), and the sign rule (closer to p^k) picks the same minimiser
    rng = np.random.default_rng(6)
    g = synth.random_graph(10, 24, seed=3)
    st = synth.random_state(rng, g.n)
    S1, S2 = _spd(rng), _spd(rng)
    st["lam"][0] = 0.0
    A1, b0 = gs.p_system(g, PARAMS, S1, S2, st, 0)
    a, V = np.linalg.eigh(A1)
    b_des = 0.3 * (a[1] - a[0]) * V[:, 1] + 0.2 * (a[2] - a[0]) * V[:, 2]
    st["lam"][0] = b0 - b_des
    A1b, b1 = gs.p_system(g, PARAMS, S1, S2, st, 0)
    _, _, hard = gs.trs_sphere(A1b, b1, st["p"][0])
    assert hard
    orc, _, nh = gs.iterate(g, PARAMS, S1, S2, st)
    assert nh >= 1
    with P.Solver(g, precision=precision) as S:
        S.set_sigma(S1, S2)
        S.set_state_full(st)
        S.step(1)
        gpu = S.state()
        fallbacks = P.pradmm_counters(S.h)["fallbacks"]
    assert np.linalg.norm(gpu["p"][0] - orc["p"][0]) <= tol
    assert relerr(gpu["p"], orc["p"]) <= tol
    if precision == 1:
        assert fallbacks >= 1


# ---- the batched form with general weights ---------------------------------------

def _walks(count, seed, n_max):
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(np.log(20), np.log(n_max), count)).round().astype(int)
    dens = rng.uniform(0.5, 3.0, count)
    return [synth.random_walk_graph(int(ns[k]), n_closures=None, closure_density=float(dens[k]), sigma_r=0.02,
                                    sigma_t=0.1, seed=3000 + k, name=f"s{k}") for k in range(count)]


@pytest.mark.parametrize("schedule", [(256, 256, 1, 0), (128, 0, 8, 50)])
def test_batch_general_sigma_matches_oracle(P, schedule):
    # FP64: every graph against the general-Sigma oracle for the iterations it
    # ran (warp/CTA items, or 8-CTA clusters above 50 poses), and the per-graph
    # objectives with the Sigma-weighted norms
    graphs = _walks(5, seed=21, n_max=300)
    rng = np.random.default_rng(22)
    S1, S2 = _spd(rng), _spd(rng)
    with P.Batch(graphs, precision=0) as B:
        B.set_sigma(S1, S2)
        B.set_schedule(*schedule)
        B.init_odometry()
        res = B.solve(rel_tol=1e-3, max_iter=40)
        st = B.state()
        F = B.objectives()
    for k, g in enumerate(graphs):
        q0, t0 = oracle.init_odometry(g)
        orc = oracle.init_state(q0, t0)
        for _ in range(int(res["iters"][k])):
            orc, _, _ = gs.iterate(g, PARAMS, S1, S2, orc)
        sl = {key: v[B.offsets[k]:B.offsets[k + 1]] for key, v in st.items()}
        for key in KEYS:
            assert relerr(sl[key], orc[key]) <= 1e-9, (k, key, relerr(sl[key], orc[key]))
        Fo = gs.objective(g, S1, S2, orc["p"], orc["t"])
        assert abs(F[k] - Fo) <= 1e-10 * max(Fo, 1.0), (k, F[k], Fo)
    conv = res["status"] == P.PRADMM_OK
    assert (res["e_last"][conv] <= 1e-3 * res["e_first"][conv]).all()


def test_batch_general_sigma_fp32_matches_single_solver(P):
    # FP32, the FP64 re-solves included: the batched form does them in the
    # sweep's own thread, the single solver in a separate kernel, from the same
    # FP32 data
    graphs = _walks(8, seed=23, n_max=3000)
    rng = np.random.default_rng(24)
    S1, S2 = _spd(rng), _spd(rng)
    with P.Batch(graphs, precision=1) as B:
        B.set_sigma(S1, S2)
        B.init_odometry()
        B.solve(rel_tol=0.0, max_iter=15)
        st = B.state()
    for k, g in enumerate(graphs):
        with P.Solver(g, precision=1) as S:
            S.set_sigma(S1, S2)
            S.init_odometry()
            S.step(15)
            ref = S.state()
        sl = {key: v[B.offsets[k]:B.offsets[k + 1]] for key, v in st.items()}
        for key in ("p", "q", "t", "s"):
            assert relerr(sl[key], ref[key]) <= 1e-5, (k, key, relerr(sl[key], ref[key]))


def test_batch_general_sigma_inertial_and_back_to_scalar(P):
    graphs = _walks(4, seed=25, n_max=200)
    rng = np.random.default_rng(26)
    S1, S2 = _spd(rng), _spd(rng)
    theta = 0.5
    with P.Batch(graphs, precision=0, inertia=theta) as B:
        B.set_sigma(S1, S2)
        B.init_odometry()
        B.solve(rel_tol=0.0, max_iter=12)
        st = B.state()
        B.set_sigma(None, None)  # scalar weights again
        B.init_odometry()
        B.solve(rel_tol=0.0, max_iter=6)
        st2 = B.state()
    for k, g in enumerate(graphs):
        q0, t0 = oracle.init_odometry(g)
        orc, prev = oracle.init_state(q0, t0), None
        for _ in range(12):
            orc, prev, _, _ = gs.iterate_inertial(g, PARAMS, S1, S2, orc, theta, prev)
        sl = {key: v[B.offsets[k]:B.offsets[k + 1]] for key, v in st.items()}
        for key in KEYS:
            assert relerr(sl[key], orc[key]) <= 1e-9, (k, key, relerr(sl[key], orc[key]))
        o2, _, _, _ = oracle.iterate_inertial(g, oracle.make_params(beta1=1.0, beta2=1.0, tau=1.5),
                                              oracle.init_state(q0, t0), theta, 6)
        sl2 = {key: v[B.offsets[k]:B.offsets[k + 1]] for key, v in st2.items()}
        for key in KEYS:
            assert relerr(sl2[key], o2[key]) <= 1e-10, (k, key)
