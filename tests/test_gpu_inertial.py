"""Inertial variant on the GPU against the oracle's inertial iteration.

Reading R27: the proximal anchors of p, q, t, s are x^k + theta (x^k - x^{k-1})
(the paper's x^{k+1/2} of Appendix B; the oracle's form is pinned in
tests/test_oracle_iteration.py).  The library keeps x^{k-1} of q, t, s in its
own arrays and takes p^{k-1} from the p double buffer; a state set restarts
the extrapolation (x^{-1} = x^0).

Tolerances as the plain parity tests: FP64 1e-10 relative per array and per
element, FP32 1e-5 for p, q, t, s and the multipliers against tau beta times
the scale they are formed from, and per element max(1e-4, 32 x the deviation
of FP32 references of the oracle's inertial iteration: executed in single
precision, and with its state and previous iterate stored in FP32); the same after a second step call (continuity of x^{k-1}).
With
general weights (pradmm_set_sigma) the general-Sigma oracle's inertial
iteration is the reference, at the general parity tolerances (FP64 1e-9, FP32
1e-4: the sphere-constrained p-update is solved by different algorithms on
the two sides).
"""
import numpy as np
import pytest

import oracle
from oracle import general_sigma as gs
from paper_2601_15684_gb300 import synth
from parity import ELEM_TOL_FP64, check_elements, check_elements_fp32, fp32_storage_run, to_fp32

pytestmark = pytest.mark.gpu
KEYS = ("p", "q", "t", "s", "lam", "z")


@pytest.fixture(scope="module")
def P():
    from paper_2601_15684_gb300 import build_lib
    from paper_2601_15684_gb300 import pradmm
    build_lib.build()
    pradmm.load()
    return pradmm


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _oparams():
    return oracle.make_params(beta1=1.0, beta2=1.0, tau=1.5, gamma=(1.0, 1e-3, 1e-3, 1e-3))


def _inertial_fp32(g, theta, st, prev, iters):
    """The oracle's inertial iteration with the state and x^{k-1} stored in FP32."""
    st = to_fp32(st)
    prev = None if prev is None else to_fp32(prev)
    for _ in range(iters):
        st, prev, _, _ = oracle.iterate_inertial(g, _oparams(), st, theta, 1, prev)
        st, prev = to_fp32(st), to_fp32(prev)
    return st, prev


def check_state(gpu, orc, fp64, what="", orc32=None):
    if fp64:
        check_elements(gpu, orc, ELEM_TOL_FP64, what=what)
    elif orc32 is not None:
        check_elements_fp32(gpu, orc, orc32, what=what)
    if fp64:
        for k in KEYS:
            assert relerr(gpu[k], orc[k]) <= 1e-10, (what, k, relerr(gpu[k], orc[k]))
        return
    for k in ("p", "q", "t", "s"):
        assert relerr(gpu[k], orc[k]) <= 1e-5, (what, k, relerr(gpu[k], orc[k]))
    assert np.linalg.norm(gpu["lam"] - orc["lam"]) <= 1e-5 * 1.5 * max(np.linalg.norm(orc["p"]), 1.0), what
    assert np.linalg.norm(gpu["z"] - orc["z"]) <= 1e-5 * 1.5 * max(np.linalg.norm(orc["t"]), 1.0), what


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("theta", [0.3, 0.7])
@pytest.mark.parametrize("case", ["ragged", "walk"])
def test_inertial_matches_oracle_one_and_ten_iterations(P, precision, theta, case):
    if case == "ragged":
        g = synth.random_graph(700, 2300, seed=41, isolated=5)
    else:
        g = synth.workload("walk128")
    st0 = synth.random_state(np.random.default_rng(7), g.n)
    with P.Solver(g, precision=precision, inertia=theta) as S:
        S.set_state_full(st0)
        orc, prev, done = st0, None, 0
        orc32, prev32 = st0, None
        orcx, prevx = st0, None
        for it in (1, 10):
            e_gpu = S.step(it - done)
            orc, prev, res, _ = oracle.iterate_inertial(g, _oparams(), orc, theta, it - done, prev)
            orc32, prev32 = _inertial_fp32(g, theta, orc32, prev32, it - done)
            orcx, prevx = oracle.iterate_inertial_f32(g, _oparams(), orcx, theta, it - done, prevx)
            done = it
            check_state(S.state(), orc, precision == 0, f"{case} theta={theta} after {it}", orc32=[orc32, orcx])
            assert abs(e_gpu - res[0]) <= (1e-9 if precision == 0 else 1e-3) * max(res[0], 1e-30)


def test_inertial_solve_stops_like_the_oracle(P):
    g = synth.workload("walk128")
    q0, t0 = oracle.init_odometry(g)
    st, prev, k, theta, tol = oracle.init_state(q0, t0), None, 0, 0.3, 1e-4
    while k < 300:
        st, prev, res, _ = oracle.iterate_inertial(g, _oparams(), st, theta, 1, prev)
        k += 1
        if res[0] < tol:
            break
    with P.Solver(g, precision=0, inertia=theta, tol=tol, max_iter=300) as S:
        S.init_odometry()
        converged, iters, e = S.solve()
        gpu = S.state()
    assert converged and iters == k
    check_state(gpu, st, True, "solve")


def test_state_set_restarts_the_extrapolation(P):
    g = synth.random_graph(300, 900, seed=5)
    st0 = synth.random_state(np.random.default_rng(3), g.n)
    theta = 0.5
    with P.Solver(g, precision=0, inertia=theta) as S:
        S.set_state_full(st0)
        S.step(4)
        mid = S.state()
        S.set_state_full(mid)  # x^{k-1} := x^k
        S.step(3)
        gpu = S.state()
    orc, _, _, _ = oracle.iterate_inertial(g, _oparams(), st0, theta, 4)
    check_state(mid, orc, True, "before restart")
    orc, _, _, _ = oracle.iterate_inertial(g, _oparams(), mid, theta, 3)  # prev = None: restart
    check_state(gpu, orc, True, "after restart")


def test_inertia_zero_is_the_plain_path(P):
    g = synth.random_graph(200, 700, seed=9)
    st0 = synth.random_state(np.random.default_rng(4), g.n)
    outs = []
    for kw in ({}, {"inertia": 0.0}):
        with P.Solver(g, precision=1, **kw) as S:
            S.set_state_full(st0)
            S.step(7)
            outs.append(S.state())
    for k in KEYS:
        np.testing.assert_array_equal(outs[0][k], outs[1][k])


def test_inertia_is_rejected_where_unsupported(P):
    g = synth.random_graph(60, 180, seed=2)
    with pytest.raises(P.PRADMMError) as ei:
        P.Solver(g, inertia=1.0)
    assert ei.value.status == P.PRADMM_ERR_ARG
    with P.Solver(g, precision=1, inertia=0.4) as S:
        S.init_odometry()


def _spd(rng, cond=8.0):
    Q, _ = np.linalg.qr(rng.normal(size=(4, 4)))
    return Q @ np.diag(np.exp(rng.uniform(0, np.log(cond), 4))) @ Q.T


GS_PARAMS = (1.0, 1.0, 1.5, (1.0, 1e-3, 1e-3, 1e-3))


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-4)])
@pytest.mark.parametrize("theta", [0.3, 0.7])
def test_inertial_general_sigma_matches_oracle(P, precision, tol, theta):
    rng = np.random.default_rng(13)
    g = synth.random_graph(97, 300, seed=5, isolated=2)
    st = synth.random_state(rng, g.n)
    S1, S2 = _spd(rng), _spd(rng)
    orc, prev = st, None
    with P.Solver(g, precision=precision, inertia=theta) as S:
        S.set_sigma(S1, S2)
        S.set_state_full(st)
        done = 0
        for it in (1, 10):
            S.step(it - done)
            for _ in range(it - done):
                orc, prev, _, _ = gs.iterate_inertial(g, GS_PARAMS, S1, S2, orc, theta, prev)
            done = it
            gpu = S.state()
            for key in ("p", "q", "t", "s"):
                assert relerr(gpu[key], orc[key]) <= tol, (it, key, relerr(gpu[key], orc[key]))
            if precision == 0:
                for key in ("lam", "z"):
                    assert relerr(gpu[key], orc[key]) <= tol, (it, key)
                check_elements(gpu, orc, tol, what=f"general theta={theta} after {it}")


def test_inertial_identity_sigma_equals_scalar_inertial_path(P):
    g = synth.random_graph(120, 360, seed=8)
    st = synth.random_state(np.random.default_rng(2), g.n)
    out = []
    for use_sigma in (False, True):
        with P.Solver(g, precision=0, inertia=0.5) as S:
            if use_sigma:
                S.set_sigma(np.eye(4), np.eye(4))
            S.set_state_full(st)
            S.step(3)
            S.step(9)
            out.append(S.state())
    for k in KEYS:
        assert relerr(out[1][k], out[0][k]) <= 1e-12, k


def test_setting_sigma_restarts_the_extrapolation(P):
    # scalar steps, then general weights: the general iterations start from
    # x^{k-1} := x^k; back to scalar weights restarts again
    rng = np.random.default_rng(17)
    g = synth.random_graph(150, 450, seed=21)
    st0 = synth.random_state(rng, g.n)
    S1, S2 = _spd(rng), _spd(rng)
    theta = 0.5
    with P.Solver(g, precision=0, inertia=theta) as S:
        S.set_state_full(st0)
        S.step(4)
        a = S.state()
        S.set_sigma(S1, S2)
        S.step(3)
        b = S.state()
        S.set_sigma(None, None)
        S.step(2)
        c = S.state()
    orc, _, _, _ = oracle.iterate_inertial(g, _oparams(), st0, theta, 4)
    check_state(a, orc, True, "scalar")
    orc, prev = a, None
    for _ in range(3):
        orc, prev, _, _ = gs.iterate_inertial(g, GS_PARAMS, S1, S2, orc, theta, prev)
    for k in KEYS:
        assert relerr(b[k], orc[k]) <= 1e-9, ("general", k, relerr(b[k], orc[k]))
    orc, _, _, _ = oracle.iterate_inertial(g, _oparams(), b, theta, 2)
    check_state(c, orc, True, "scalar again")


def _walks(count, seed, n_max):
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(np.log(20), np.log(n_max), count)).round().astype(int)
    dens = rng.uniform(0.5, 3.0, count)
    return [synth.random_walk_graph(int(ns[k]), n_closures=None, closure_density=float(dens[k]), sigma_r=0.02,
                                    sigma_t=0.1, seed=2000 + k, name=f"w{k}") for k in range(count)]


@pytest.mark.parametrize("schedule", [(256, 256, 1, 0), (128, 0, 8, 50)])
def test_batch_inertial_matches_oracle_graph_by_graph(P, schedule):
    # every graph of the batch runs its own inertial iteration (warp, CTA or
    # cluster groups) and stops by the batch's relative rule; a second solve
    # starts the extrapolation afresh from the first one's result
    graphs = _walks(6, seed=11, n_max=400)
    theta = 0.4
    with P.Batch(graphs, precision=0, inertia=theta) as B:
        B.set_schedule(*schedule)
        B.init_odometry()
        res = B.solve(rel_tol=1e-3, max_iter=60)
        first = B.state()
        B.solve(rel_tol=0.0, max_iter=5)
        second = B.state()
    for k, g in enumerate(graphs):
        q0, t0 = oracle.init_odometry(g)
        orc, _, _, _ = oracle.iterate_inertial(g, _oparams(), oracle.init_state(q0, t0), theta, int(res["iters"][k]))
        sl = {key: v[B.offsets[k]:B.offsets[k + 1]] for key, v in first.items()}
        check_state(sl, orc, True, f"graph {k}")
        orc, _, _, _ = oracle.iterate_inertial(g, _oparams(), sl, theta, 5)
        sl2 = {key: v[B.offsets[k]:B.offsets[k + 1]] for key, v in second.items()}
        check_state(sl2, orc, True, f"graph {k}, second solve")
    conv = res["status"] == P.PRADMM_OK
    assert (res["e_last"][conv] <= 1e-3 * res["e_first"][conv]).all()


def test_batch_inertial_fp32_matches_single_solver(P):
    graphs = _walks(10, seed=12, n_max=2500)
    theta = 0.3
    with P.Batch(graphs, precision=1, inertia=theta) as B:
        B.init_odometry()
        B.solve(rel_tol=0.0, max_iter=20)
        st = B.state()
    for k, g in enumerate(graphs):
        with P.Solver(g, precision=1, inertia=theta) as S:
            S.init_odometry()
            S.step(20)
            ref = S.state()
        sl = {key: v[B.offsets[k]:B.offsets[k + 1]] for key, v in st.items()}
        # p, q, t, s at 1e-5; the multipliers are running sums of one rounded
        # increment per iteration: 1e-5 sqrt(iterations) of the scale they are
        # formed from (the batched form's tolerance)
        for key in ("p", "q", "t", "s"):
            assert relerr(sl[key], ref[key]) <= 1e-5, (k, key, relerr(sl[key], ref[key]))
        grow = np.sqrt(20.0)
        assert np.linalg.norm(sl["lam"] - ref["lam"]) <= 1e-5 * grow * 1.5 * max(np.linalg.norm(ref["p"]), 1.0), k
        assert np.linalg.norm(sl["z"] - ref["z"]) <= 1e-5 * grow * 1.5 * max(np.linalg.norm(ref["t"]), 1.0), k


# ---- reverse mode of the inertial iteration ------------------------------------
# Against the oracle's inertial reverse mode (pinned by central differences),
# per gradient array: FP64 1e-8, FP32 1e-3, as the plain reverse-mode tests.

@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-3)])
@pytest.mark.parametrize("theta", [0.4, 0.8])
def test_inertial_reverse_mode_matches_oracle(P, precision, tol, theta):
    g = synth.random_graph(240, 700, seed=44, isolated=3)
    st = synth.random_state(np.random.default_rng(12), g.n)
    rng = np.random.default_rng(13)
    pb, tb = rng.normal(size=(g.n, 4)), rng.normal(size=(g.n, 3))
    K = 17
    prm = oracle.make_params(beta1=1.0, beta2=1.0, tau=1.5, gamma=(1.0, 0.6, 0.5, 0.7))
    ref = oracle.adjoint_inertial(g, prm, st, K, theta, pb, tb)
    with P.Solver(g, precision=precision, inertia=theta, gamma=(1.0, 0.6, 0.5, 0.7)) as S:
        S.set_state_full(st)
        S.adjoint_record(K, 0)
        assert S.adjoint_tape_info()[0] == 1
        fin = S.state()
        got = S.adjoint(pb, tb, x0=True)
    for key in ("q_meas", "t_meas", "kappa", "omega"):
        assert relerr(got[key], ref[key]) <= tol, (key, relerr(got[key], ref[key]))
    for key in KEYS:
        assert relerr(got["x0"][key], ref["x0"][key]) <= tol, ("x0", key, relerr(got["x0"][key], ref["x0"][key]))
    assert relerr(fin["p"], ref["p"]) <= (1e-10 if precision == 0 else 1e-4)


def test_inertial_record_restarts_the_extrapolation(P):
    # a record after steps starts from the current state with x^{-1} = x^0
    g = synth.random_graph(150, 420, seed=45)
    st = synth.random_state(np.random.default_rng(14), g.n)
    theta = 0.5
    with P.Solver(g, precision=0, inertia=theta) as S:
        S.set_state_full(st)
        S.step(4)
        mid = S.state()
        S.adjoint_record(6, 1)
        fin = S.state()
    orc, _, _, _ = oracle.iterate_inertial(g, _oparams(), mid, theta, 6)
    check_state(fin, orc, True, "recorded")


def test_inertial_degenerate_graphs(P):
    # no edges (n = 1 and 5), and a vertex whose u is 0 in the first
    # iteration (its p is kept, as in the plain iteration)
    theta = 0.5
    for n in (1, 5):
        g = synth.PoseGraph(n=n, src=np.zeros(0, np.int32), dst=np.zeros(0, np.int32), q_meas=np.zeros((0, 4)),
                            t_meas=np.zeros((0, 3)), kappa=np.zeros(0), omega=np.zeros(0))
        st0 = synth.random_state(np.random.default_rng(n), n)
        for precision in (0, 1):
            with P.Solver(g, precision=precision, inertia=theta) as S:
                S.set_state_full(st0)
                S.step(1)
                S.step(3)
                gpu = S.state()
            orc, _, _, _ = oracle.iterate_inertial(g, _oparams(), st0, theta, 4)
            check_state(gpu, orc, precision == 0, f"n={n}")
    g = synth.random_graph(6, 10, seed=31, isolated=1)
    st = synth.random_state(np.random.default_rng(32), g.n)
    st["p"][5] = st["q"][5] = [1.0, 0, 0, 0]
    st["lam"][5] = [-2.0, 0, 0, 0]
    with P.Solver(g, precision=0, inertia=theta) as S:
        S.set_state_full(st)
        S.step(1)
        assert S.counters()["zero_u"] == 1
        gpu = S.state()
    np.testing.assert_array_equal(gpu["p"][5], [1.0, 0, 0, 0])
    orc, _, _, _ = oracle.iterate_inertial(g, _oparams(), st, theta, 1)
    check_state(gpu, orc, True, "zero u")


@pytest.mark.parametrize("K", [0, 1, 2])
def test_inertial_reverse_mode_short_tapes(P, K):
    g = synth.random_graph(60, 170, seed=46, isolated=2)
    st = synth.random_state(np.random.default_rng(15), g.n)
    rng = np.random.default_rng(16)
    pb, tb = rng.normal(size=(g.n, 4)), rng.normal(size=(g.n, 3))
    prm = oracle.make_params(beta1=1.0, beta2=1.0, tau=1.5, gamma=(1.0, 0.6, 0.5, 0.7))
    ref = oracle.adjoint_inertial(g, prm, st, K, 0.6, pb, tb)
    with P.Solver(g, precision=0, inertia=0.6, gamma=(1.0, 0.6, 0.5, 0.7)) as S:
        S.set_state_full(st)
        S.adjoint_record(K, 1)
        got = S.adjoint(pb, tb, x0=True)
    for key in ("q_meas", "t_meas", "kappa", "omega"):
        if K == 0:
            assert not np.any(got[key])
        else:
            assert relerr(got[key], ref[key]) <= 1e-8, (key, relerr(got[key], ref[key]))
    for key in KEYS:
        if np.linalg.norm(ref["x0"][key]) == 0.0:
            assert not np.any(got["x0"][key]), key
        else:
            assert relerr(got["x0"][key], ref["x0"][key]) <= 1e-8, ("x0", key)


def test_inertial_checkpoint_spacing_is_bitwise_irrelevant(P):
    # checkpoints carry x^{k-1} (q, t, s and p), so every spacing recomputes
    # the same iterates and gives bitwise the same gradients
    g = synth.random_graph(180, 520, seed=47)
    st = synth.random_state(np.random.default_rng(17), g.n)
    rng = np.random.default_rng(18)
    pb, tb = rng.normal(size=(g.n, 4)), rng.normal(size=(g.n, 3))
    outs = []
    for ckpt in (1, 3, 7, 23, 0):
        with P.Solver(g, precision=1, inertia=0.5, gamma=(1.0, 0.6, 0.5, 0.7)) as S:
            S.set_state_full(st)
            S.adjoint_record(23, ckpt)
            outs.append(S.adjoint(pb, tb, x0=True))
    for o in outs[1:]:
        for key in ("q_meas", "t_meas", "kappa", "omega"):
            np.testing.assert_array_equal(o[key], outs[0][key])
        for key in KEYS:
            np.testing.assert_array_equal(o["x0"][key], outs[0]["x0"][key])
    prm = oracle.make_params(beta1=1.0, beta2=1.0, tau=1.5, gamma=(1.0, 0.6, 0.5, 0.7))
    ref = oracle.adjoint_inertial(g, prm, st, 23, 0.5, pb, tb)
    for key in ("q_meas", "t_meas", "kappa", "omega"):
        assert relerr(outs[0][key], ref[key]) <= 1e-3, key
