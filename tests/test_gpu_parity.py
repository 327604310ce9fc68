"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every comparison with the oracle is made per array and element by element
(tests/parity.py: per vertex |X_gpu,i - X_orc,i| / max(|X_orc,i|, floor)):
FP64 every element within ELEM_TOL_FP64 = 1e-10; FP32 every element within
max(1e-4, 32 x the deviation at the vertex of FP32 references from the same
start -- the checker's algorithm executed in single precision and the FP64
oracle with its state stored in FP32 --, 32 x their root mean square
deviation).

Tolerances (relerr(X) = |X_gpu - X_oracle|_2 / |X_oracle|_2 per state array):
  FP64 path: 1e-10 after 1 and 10 iterations (rounding-order differences only;
             measured ~1e-15), final objective within 1e-6 relative.
  FP32 path: p, q, t, s within 1e-5 relative after 1 and 10 iterations.  The
             multipliers are sums of tau*beta*(p - q) and tau*beta*(t - s),
             differences of nearly equal stored values, so their error is
             measured against the scale they are formed from:
             |dlam| <= 1e-5 * tau*beta1*|p|,  |dz| <= 1e-5 * tau*beta2*|t|
             (FP32 unit roundoff 6e-8 times the few-term sums of one update,
             with margin).
"""
import numpy as np
import pytest

import oracle
from paper_2601_15684_gb300 import synth
from parity import ELEM_TOL_FP64, check_elements, check_elements_fp32, fp32_storage_run

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


def _params(P, precision, beta1=1.0, beta2=1.0, tau=1.5, gamma=(1.0, 1e-3, 1e-3, 1e-3), use_graph=1, block=0,
            tol=1e-4, max_iter=300):
    prm = P.pradmm_default_params()
    prm.beta1, prm.beta2, prm.relax = beta1, beta2, tau
    for k in range(4):
        prm.gamma[k] = gamma[k]
    prm.precision = precision
    prm.use_graph = use_graph
    prm.block = block
    prm.tol = tol
    prm.max_iter = max_iter
    return prm


def _oparams(beta1=1.0, beta2=1.0, tau=1.5, gamma=(1.0, 1e-3, 1e-3, 1e-3)):
    return oracle.make_params(beta1=beta1, beta2=beta2, tau=tau, gamma=gamma)


def check_state(gpu, orc, fp64, prm, what="", orc32=None):
    """orc: the FP64 oracle's state; orc32 (FP32 path): the FP32 reference
    states for the same iterations, for the per-element rule (None when
    comparing two GPU runs: per-array bounds only)."""
    if fp64:
        check_elements(gpu, orc, ELEM_TOL_FP64, what=what, tau=prm.relax, beta1=prm.beta1, beta2=prm.beta2)
    elif orc32 is not None:
        check_elements_fp32(gpu, orc, orc32, what=what, tau=prm.relax, beta1=prm.beta1, beta2=prm.beta2)
    if fp64:
        for k in KEYS:
            assert relerr(gpu[k], orc[k]) <= 1e-10, (k, relerr(gpu[k], orc[k]))
        return
    for k in ("p", "q", "t", "s"):
        assert relerr(gpu[k], orc[k]) <= 1e-5, (k, relerr(gpu[k], orc[k]))
    assert np.linalg.norm(gpu["lam"] - orc["lam"]) <= 1e-5 * prm.relax * prm.beta1 * np.linalg.norm(orc["p"])
    assert np.linalg.norm(gpu["z"] - orc["z"]) <= 1e-5 * prm.relax * prm.beta2 * np.linalg.norm(orc["t"])


def _run_pair(P, g, st0, prm, iters_list=(1, 10)):
    op = _oparams(prm.beta1, prm.beta2, prm.relax, tuple(prm.gamma))
    step = lambda st: oracle.iterate(g, op, st, 1)[0]
    with P.Solver(g, prm) as S:
        S.set_state_full(st0)
        done = 0
        orc = st0
        orc32, orcx = st0, st0
        for it in iters_list:
            e_gpu = S.step(it - done)
            orc, res, _ = oracle.iterate(g, op, orc, it - done)
            orc32 = fp32_storage_run(step, orc32, it - done)
            orcx = oracle.iterate_f32(g, op, orcx, it - done)
            done = it
            gpu = S.state()
            check_state(gpu, orc, prm.precision == P.PRADMM_FP64, prm, what=f"{g.name or g.n} after {it}",
                        orc32=[orc32, orcx])
            assert abs(e_gpu - res[0]) <= (1e-9 if prm.precision == P.PRADMM_FP64 else 1e-3) * max(res[0], 1e-30)
            assert S.iterations() == it


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", ["ragged", "hubs", "isolated", "tail"])
def test_random_graphs_one_and_ten_iterations(P, precision, case):
    if case == "ragged":
        g = synth.random_graph(3000, 9000, seed=1)
    elif case == "hubs":
        g = synth.random_graph(700, 6000, seed=2)  # pareto-skewed tails: high-degree hubs
    elif case == "isolated":
        g = synth.random_graph(1200, 2500, seed=3, isolated=300)
    else:
        g = synth.random_graph(257, 700, seed=4)  # one vertex past a 256-thread CTA
    st0 = synth.random_state(np.random.default_rng(10), g.n)
    prm = _params(P, precision, beta1=3.0, beta2=5.0, tau=1.3, gamma=(0.7, 0.01, 0.02, 0.03))
    _run_pair(P, g, st0, prm)


@pytest.mark.parametrize("precision", [0, 1])
def test_walk128_odometry_and_iterates(P, precision):
    g = synth.workload("walk128")
    prm = _params(P, precision)
    q0, t0 = oracle.init_odometry(g)
    with P.Solver(g, prm) as S:
        S.init_odometry()
        st = S.state()
        tq = 1e-12 if precision == 0 else 1e-6
        tt = 1e-10 if precision == 0 else 1e-6 * max(1.0, np.abs(t0).max())
        assert np.abs(st["q"] - q0).max() < tq
        assert np.abs(st["t"] - t0).max() < tt
    _run_pair(P, g, oracle.init_state(q0, t0), prm)


def test_walk128_fp64_solve_500_objective(P):
    """Config: 128-pose walk, FP64, 500 iterations; final objective within 1e-6."""
    g = synth.workload("walk128")
    prm = _params(P, 0)
    q0, t0 = oracle.init_odometry(g)
    with P.Solver(g, prm) as S:
        S.set_state(q0, t0)
        S.step(500)
        F_gpu = S.objective()
        gpu = S.state()
    orc, _, _ = oracle.iterate(g, _oparams(), oracle.init_state(q0, t0), 500)
    F_orc = oracle.objective(g, orc["p"], orc["t"])
    assert abs(F_gpu - F_orc) <= 1e-6 * F_orc
    assert abs(oracle.objective(g, gpu["p"], gpu["t"]) - F_gpu) <= 1e-12 * F_orc
    for k in KEYS:
        assert relerr(gpu[k], orc[k]) <= 1e-8, k
    check_elements(gpu, orc, 1e-8, what="walk128 FP64 after 500")


def test_solve_stops_like_the_oracle(P):
    g = synth.workload("walk128")
    prm = _params(P, 0, tol=3e-4, max_iter=400)
    q0, t0 = oracle.init_odometry(g)
    orc, k_orc, e_orc, trace = oracle.solve(g, _oparams(), oracle.init_state(q0, t0), 400, 3e-4)
    assert k_orc < 400 and abs(trace[k_orc - 2] - 3e-4) > 1e-8  # not a borderline crossing
    for use_graph in (1, 0):
        prm.use_graph = use_graph
        with P.Solver(g, prm) as S:
            S.set_state(q0, t0)
            conv, k, e = S.solve()
            assert conv and k == k_orc
            assert abs(e - e_orc) <= 1e-9 * e_orc
            gpu = S.state()
            for key in KEYS:
                assert relerr(gpu[key], orc[key]) <= 1e-10, key
            check_elements(gpu, orc, ELEM_TOL_FP64, what=f"solve stopped at {k}")


def test_solve_not_converged_keeps_state(P):
    g = synth.workload("walk128")
    prm = _params(P, 0, tol=1e-30, max_iter=7)
    q0, t0 = oracle.init_odometry(g)
    with P.Solver(g, prm) as S:
        S.set_state(q0, t0)
        conv, k, e = S.solve()
        assert not conv and k == 7 and S.iterations() == 7
        orc, res, _ = oracle.iterate(g, _oparams(), oracle.init_state(q0, t0), 7)
        for key in KEYS:
            assert relerr(S.state()[key], orc[key]) <= 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_and_plain_launches_bit_identical_and_deterministic(P, precision):
    g = synth.random_graph(5000, 20000, seed=7)
    st0 = synth.random_state(np.random.default_rng(8), g.n)
    outs = []
    for use_graph in (1, 0, 1):
        prm = _params(P, precision, use_graph=use_graph)
        with P.Solver(g, prm) as S:
            S.set_state_full(st0)
            e = S.step(6)
            outs.append((e, S.state(), S.objective()))
    for e, st, F in outs[1:]:
        assert e == outs[0][0] and F == outs[0][2]
        for k in KEYS:
            np.testing.assert_array_equal(st[k], outs[0][1][k])


def test_checkpoint_resume_matches_uninterrupted(P):
    g = synth.workload("helix25k")
    prm = _params(P, 1)
    q0, t0 = oracle.init_odometry(g)
    with P.Solver(g, prm) as A:
        A.set_state(q0, t0)
        A.step(20)
        full = A.state()
    with P.Solver(g, prm) as B:
        B.set_state(q0, t0)
        B.step(8)
        ck = B.state()
    with P.Solver(g, prm) as C:
        C.set_state_full(ck)
        C.step(12)
        res = C.state()
    # the checkpoint round-trips exactly (FP32 values through double); the
    # resumed run recomputes the first p-block directly where the
    # uninterrupted run folded it into the s sweep, so the two agree to FP32
    # rounding (the FP32 parity bound) rather than bitwise
    check_state(res, full, False, prm)


def test_block_sizes_agree(P):
    g = synth.random_graph(4000, 12000, seed=9, isolated=7)
    st0 = synth.random_state(np.random.default_rng(3), g.n)
    ref = None
    for block in (32, 96, 256):
        prm = _params(P, 0, block=block)
        with P.Solver(g, prm) as S:
            S.set_state_full(st0)
            S.step(3)
            st = S.state()
        if ref is None:
            ref = st
        for k in KEYS:
            assert relerr(st[k], ref[k]) <= 1e-13


def test_edge_cases(P):
    # no edges at all: every vertex is isolated; n = 1
    for n in (1, 5):
        g = synth.PoseGraph(n=n, src=np.zeros(0, np.int32), dst=np.zeros(0, np.int32), q_meas=np.zeros((0, 4)),
                            t_meas=np.zeros((0, 3)), kappa=np.zeros(0), omega=np.zeros(0))
        st0 = synth.random_state(np.random.default_rng(n), n)
        for precision in (0, 1):
            prm = _params(P, precision)
            with P.Solver(g, prm) as S:
                S.set_state_full(st0)
                S.step(4)
                gpu = S.state()
                assert S.objective() == 0.0
            orc, _, _ = oracle.iterate(g, _oparams(), st0, 4)
            orc32 = [fp32_storage_run(lambda st: oracle.iterate(g, _oparams(), st, 1)[0], st0, 4),
                     oracle.iterate_f32(g, _oparams(), st0, 4)]
            check_state(gpu, orc, precision == 0, prm, what=f"no edges, n={n}", orc32=orc32)
    # |u| = 0 keeps p (reading of the undefined normalisation)
    g = synth.random_graph(6, 10, seed=31, isolated=1)
    st = synth.random_state(np.random.default_rng(32), g.n)
    st["p"][5] = st["q"][5] = [1.0, 0, 0, 0]
    st["lam"][5] = [-2.0, 0, 0, 0]
    for precision in (0, 1):
        with P.Solver(g, _params(P, precision)) as S:
            S.set_state_full(st)
            S.step(1)
            c = S.counters()
            assert c["zero_u"] == 1
            assert c["fallbacks"] == (1 if precision == 1 else 0)
            np.testing.assert_array_equal(S.state()["p"][5], [1.0, 0, 0, 0])


def test_input_errors(P):
    g = synth.random_graph(10, 20, seed=5)
    bad = [
        dict(dst=np.where(np.arange(20) == 3, 10, g.dst)),  # out of range
        dict(dst=np.where(np.arange(20) == 3, g.src, g.dst)),  # self-loop
    ]
    codes = [P.PRADMM_ERR_INDEX, P.PRADMM_ERR_SELFLOOP]
    for kw, code in zip(bad, codes):
        with pytest.raises(P.PRADMMError) as ei:
            P.pradmm_create(g.n, kw.get("src", g.src), kw["dst"], g.q_meas, g.t_meas)
        assert ei.value.status == code
    qm = g.q_meas.copy()
    qm[2] *= 1.01
    with pytest.raises(P.PRADMMError) as ei:
        P.pradmm_create(g.n, g.src, g.dst, qm, g.t_meas)
    assert ei.value.status == P.PRADMM_ERR_QUATERNION
    tm = g.t_meas.copy()
    tm[4, 1] = np.nan
    with pytest.raises(P.PRADMMError) as ei:
        P.pradmm_create(g.n, g.src, g.dst, g.q_meas, tm)
    assert ei.value.status == P.PRADMM_ERR_NONFINITE
    prm = _params(P, 1, tau=2.0)
    with pytest.raises(P.PRADMMError) as ei:
        P.pradmm_create(g.n, g.src, g.dst, g.q_meas, g.t_meas, params=prm)
    assert ei.value.status == P.PRADMM_ERR_ARG
    h = P.pradmm_create(g.n, g.src, g.dst, g.q_meas, g.t_meas)
    try:
        with pytest.raises(P.PRADMMError) as ei:
            P.pradmm_step(h, 1)
        assert ei.value.status == P.PRADMM_ERR_STATE
    finally:
        P.pradmm_destroy(h)


def test_input_errors_in_a_large_edge_list_name_the_first_bad_edge(P):
    # the edges are validated on the device (every edge by its own thread);
    # the error must still be the first invalid edge in input order, with
    # the message the host forms for it
    g = synth.random_graph(50000, 200000, seed=8)
    cases = [
        ("dst", {170000: 50000, 150001: -1}, P.PRADMM_ERR_INDEX, "edge 150001"),
        ("dst", {199999: -3, 120000: "self"}, P.PRADMM_ERR_SELFLOOP, "edge 120000"),
    ]
    for field, bad, code, text in cases:
        dst = g.dst.copy()
        for e, v in bad.items():
            dst[e] = g.src[e] if v == "self" else v
        with pytest.raises(P.PRADMMError) as ei:
            P.pradmm_create(g.n, g.src, dst, g.q_meas, g.t_meas)
        assert ei.value.status == code
        assert text in str(ei.value), str(ei.value)
    qm = g.q_meas.copy()
    qm[180000] *= 1.5
    qm[160000, 2] = np.nan
    with pytest.raises(P.PRADMMError) as ei:
        P.pradmm_create(g.n, g.src, g.dst, qm, g.t_meas)
    assert ei.value.status == P.PRADMM_ERR_NONFINITE and "edge 160000" in str(ei.value)


def test_input_validation_boundaries(P):
    """The device validation takes the host's decisions: |q_e| accepted within
    1e-6 of 1 (squared norm summed in component order with separate
    roundings, then the square root), weights finite and > 0."""
    import math

    g = synth.random_graph(40, 100, seed=12)
    for scale in (1 + 0.5e-6, 1 + 0.999e-6, 1 + 1.001e-6, 1 - 0.999e-6, 1 - 1.001e-6, 1 + 3e-6):
        qm = g.q_meas.copy()
        qm[7] *= scale
        q = [float(x) for x in qm[7]]
        nn = 0.0
        for x in q:
            nn = nn + x * x
        ok = abs(math.sqrt(nn) - 1.0) <= 1e-6
        if ok:
            P.pradmm_destroy(P.pradmm_create(g.n, g.src, g.dst, qm, g.t_meas))
        else:
            with pytest.raises(P.PRADMMError) as ei:
                P.pradmm_create(g.n, g.src, g.dst, qm, g.t_meas)
            assert ei.value.status == P.PRADMM_ERR_QUATERNION and "edge 7" in str(ei.value), str(ei.value)
    for name, val, code in (("kappa", 0.0, P.PRADMM_ERR_ARG), ("kappa", -1.0, P.PRADMM_ERR_ARG),
                            ("omega", np.inf, P.PRADMM_ERR_NONFINITE), ("omega", np.nan, P.PRADMM_ERR_NONFINITE),
                            ("kappa", -np.inf, P.PRADMM_ERR_NONFINITE)):
        ka, om = g.kappa.copy(), g.omega.copy()
        (ka if name == "kappa" else om)[11] = val
        with pytest.raises(P.PRADMMError) as ei:
            P.pradmm_create(g.n, g.src, g.dst, g.q_meas, g.t_meas, ka, om)
        assert ei.value.status == code and "edge 11" in str(ei.value), (name, val, str(ei.value))


def test_nonfinite_state_is_reported(P):
    g = synth.random_graph(50, 120, seed=6)
    st = synth.random_state(np.random.default_rng(6), g.n)
    with P.Solver(g, _params(P, 1)) as S:
        st["t"][3] = 3.3e38  # finite inputs whose products overflow FP32
        st["s"][3] = 3.3e38
        S.set_state_full(st)
        with pytest.raises(P.PRADMMError) as ei:
            S.step(3)
        assert ei.value.status == P.PRADMM_ERR_NONFINITE


@pytest.mark.parametrize("precision", [0, 1])
def test_autotune_picks_a_cta_size_and_restores_the_state(P, precision):
    g = synth.random_graph(5000, 15000, seed=51, isolated=4)
    st0 = synth.random_state(np.random.default_rng(52), g.n)
    with P.Solver(g, _params(P, precision)) as S:
        S.set_state_full(st0)
        before = S.state()
        blk = S.autotune(8)
        assert blk in (32, 64, 128, 256)
        after = S.state()
        assert S.iterations() == 0
        for k in KEYS:
            np.testing.assert_array_equal(after[k], before[k])
        S.step(5)
        tuned = S.state()
    with P.Solver(g, _params(P, precision, block=blk)) as S:
        S.set_state_full(st0)
        S.step(5)
        ref = S.state()
    for k in KEYS:
        assert relerr(tuned[k], ref[k]) <= (1e-13 if precision == 0 else 1e-6), k
    orc, _, _ = oracle.iterate(g, _oparams(), st0, 5)
    orc32 = [fp32_storage_run(lambda st: oracle.iterate(g, _oparams(), st, 1)[0], st0, 5),
             oracle.iterate_f32(g, _oparams(), st0, 5)]
    check_state(tuned, orc, precision == 0, _params(P, precision), what="autotuned", orc32=orc32)


@pytest.mark.parametrize("precision", [0, 1])
def test_residual_trace_matches_the_oracle(P, precision):
    # the device ring of e^k (Appendix E.1): every iteration of a solve, in
    # order, against the oracle's own residuals; a wrapped ring keeps the last
    # `capacity`; a state set restarts it; the reverse pass's replays do not
    # write it
    g = synth.workload("walk128")
    q0, t0 = oracle.init_odometry(g)
    _, k_orc, _, trace = oracle.solve(g, _oparams(), oracle.init_state(q0, t0), 120, 0.0)
    tol = 1e-9 if precision == 0 else 2e-3
    with P.Solver(g, _params(P, precision)) as S:
        S.set_trace(50)
        S.set_state(q0, t0)
        S.step(30)
        first, e = S.trace()
        assert first == 1 and e.size == 30
        np.testing.assert_allclose(e, trace[:30], rtol=tol)
        S.step(90)
        first, e = S.trace()
        assert first == 71 and e.size == 50
        np.testing.assert_allclose(e, trace[70:120], rtol=tol)
        S.set_state(q0, t0)
        S.adjoint_record(10, 3)
        S.adjoint(np.ones((g.n, 4)), np.ones((g.n, 3)))
        first, e = S.trace()
        assert first == 1 and e.size == 10
        np.testing.assert_allclose(e, trace[:10], rtol=tol)
        S.set_trace(0)
        with pytest.raises(P.PRADMMError) as ei:
            S.trace()
        assert ei.value.status == P.PRADMM_ERR_STATE
