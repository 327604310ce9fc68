"""Reverse mode on the GPU against the oracle's reverse mode.

The oracle's adjoint is itself pinned by central finite differences
(test_oracle_adjoint.py).  Here the CUDA adjoint (pradmm_adjoint_record +
pradmm_adjoint) must give the same gradients, per output array
relerr = |g_gpu - g_oracle|_2 / |g_oracle|_2:
  FP64 path: <= 1e-8   (rounding order only; the reverse sweeps sum in a
                        different order than the oracle's edge loops)
  FP32 path: <= 1e-3   (state and reverse sweeps in FP32; gradients summed in
                        FP64 across iterations)
On the FP64 path every row (an edge's or a vertex's gradient) is also held
to 1e-8 of the larger of its own norm and the root mean square row norm of
the oracle's array.
Checkpointing must not change anything: segments are recomputed with the
forward kernels, so every ckpt_every gives bitwise the same gradients.
"""
import numpy as np
import pytest

import oracle
from oracle.anchor import anchor_loss as anchor_loss_np
from paper_2601_15684_gb300 import synth

pytestmark = pytest.mark.gpu
GRADS = ("q_meas", "t_meas", "kappa", "omega")
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


def row_err(a, b):
    """Largest row error |a_r - b_r| over max(|b_r|, rms_r |b_r|)."""
    a = np.asarray(a).reshape(len(a), -1)
    b = np.asarray(b).reshape(len(b), -1)
    if len(b) == 0:
        return 0.0
    nb = np.linalg.norm(b, axis=1)
    scale = np.maximum(nb, np.sqrt(np.mean(nb * nb)))
    return float(np.max(np.linalg.norm(a - b, axis=1) / np.maximum(scale, 1e-300)))


def _oparams():
    return oracle.make_params(beta1=1.0, beta2=1.0, tau=1.5, gamma=(1.0, 1e-3, 1e-3, 1e-3))


def _cotangent(n, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, 4)), rng.normal(size=(n, 3))


def _gpu_adjoint(P, g, st, K, pb, tb, precision, ckpt=7, x0=True):
    with P.Solver(g, precision=precision) as S:
        S.set_state_full(st)
        S.adjoint_record(K, ckpt)
        fin = S.state()
        out = S.adjoint(pb, tb, x0=x0)
    out["final"] = fin
    return out


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-3)])
@pytest.mark.parametrize("shape", [(300, 900, 30), (97, 250, 13)])
def test_adjoint_matches_oracle(P, precision, tol, shape):
    n, m, K = shape
    g = synth.random_graph(n, m, seed=n + m, isolated=3)
    st = synth.random_state(np.random.default_rng(n), n)
    pb, tb = _cotangent(n, 1)
    ref = oracle.adjoint(g, _oparams(), st, K, pb, tb)
    got = _gpu_adjoint(P, g, st, K, pb, tb, precision)
    for key in GRADS:
        assert relerr(got[key], ref[key]) <= tol, (key, relerr(got[key], ref[key]))
    for key in KEYS:
        assert relerr(got["x0"][key], ref["x0"][key]) <= tol, ("x0", key, relerr(got["x0"][key], ref["x0"][key]))
    if precision == 0:
        for key in GRADS:
            r = row_err(got[key], ref[key])
            print(f"{shape} {key}: largest row error {r:.3e}")
            assert r <= tol, (key, r)
        for key in KEYS:
            r = row_err(got["x0"][key], ref["x0"][key])
            print(f"{shape} x0 {key}: largest row error {r:.3e}")
            assert r <= tol, ("x0", key, r)
    # the recorded forward is the plain forward
    assert relerr(got["final"]["p"], ref["p"]) <= (1e-10 if precision == 0 else 1e-4)


def test_checkpoint_spacing_is_bitwise_irrelevant(P):
    g = synth.random_graph(200, 600, seed=5)
    st = synth.random_state(np.random.default_rng(2), g.n)
    pb, tb = _cotangent(g.n, 3)
    outs = [_gpu_adjoint(P, g, st, 23, pb, tb, 1, ckpt=c) for c in (1, 4, 7, 23, 100, 0)]
    for o in outs[1:]:
        for key in GRADS:
            np.testing.assert_array_equal(o[key], outs[0][key])
        for key in KEYS:
            np.testing.assert_array_equal(o["x0"][key], outs[0]["x0"][key])


def test_adjoint_is_linear_and_repeatable(P):
    g = synth.random_graph(150, 400, seed=9)
    st = synth.random_state(np.random.default_rng(4), g.n)
    a_p, a_t = _cotangent(g.n, 5)
    b_p, b_t = _cotangent(g.n, 6)
    with P.Solver(g, precision=0) as S:
        S.set_state_full(st)
        S.adjoint_record(15, 4)
        ga = S.adjoint(a_p, a_t)
        gb = S.adjoint(b_p, b_t)
        gab = S.adjoint(a_p + 2 * b_p, a_t + 2 * b_t)
        ga2 = S.adjoint(a_p, a_t)
        gp_only = S.adjoint(a_p, None)
        gt_only = S.adjoint(None, a_t)
    for key in GRADS:
        np.testing.assert_array_equal(ga[key], ga2[key])
        assert relerr(gab[key], ga[key] + 2 * gb[key]) <= 1e-12
        assert relerr(gp_only[key] + gt_only[key], ga[key]) <= 1e-12


def test_zero_iterations_returns_cotangent(P):
    g = synth.random_graph(40, 100, seed=1)
    st = synth.random_state(np.random.default_rng(0), g.n)
    pb, tb = _cotangent(g.n, 2)
    got = _gpu_adjoint(P, g, st, 0, pb, tb, 0, ckpt=5)
    for key in GRADS:
        assert not got[key].any()
    np.testing.assert_array_equal(got["x0"]["p"], pb)
    np.testing.assert_array_equal(got["x0"]["t"], tb)
    for key in ("q", "s", "lam", "z"):
        assert not got["x0"][key].any()


def test_tape_is_invalidated_by_state_changes(P):
    g = synth.random_graph(40, 100, seed=2)
    st = synth.random_state(np.random.default_rng(1), g.n)
    pb, tb = _cotangent(g.n, 2)
    with P.Solver(g, precision=1) as S:
        with pytest.raises(P.PRADMMError) as ei:
            S.adjoint(pb, tb)
        assert ei.value.status == P.PRADMM_ERR_STATE
        S.set_state_full(st)
        S.adjoint_record(5, 2)
        S.adjoint(pb, tb)
        S.step(1)
        with pytest.raises(P.PRADMMError) as ei:
            S.adjoint(pb, tb)
        assert ei.value.status == P.PRADMM_ERR_STATE
        S.adjoint_record(5, 2)
        S.adjoint(pb, tb)
        S.set_state_full(st)
        with pytest.raises(P.PRADMMError):
            S.adjoint(pb, tb)
        with pytest.raises(P.PRADMMError) as ei:
            S.adjoint_record(5, -1)
        assert ei.value.status == P.PRADMM_ERR_ARG
        with pytest.raises(P.PRADMMError) as ei:
            S.adjoint_tape_info()
        assert ei.value.status == P.PRADMM_ERR_STATE


def test_adjoint_after_steps_uses_current_state(P):
    # recording from x^k (k > 0, odd) keeps the p double buffer's parity
    g = synth.random_graph(120, 360, seed=12)
    st = synth.random_state(np.random.default_rng(7), g.n)
    pb, tb = _cotangent(g.n, 8)
    with P.Solver(g, precision=0) as S:
        S.set_state_full(st)
        S.step(3)
        mid = S.state()
        S.adjoint_record(9, 4)
        got = S.adjoint(pb, tb, x0=True)
    xk, _, _ = oracle.iterate(g, _oparams(), st, 3)
    ref = oracle.adjoint(g, _oparams(), xk, 9, pb, tb)
    for key in GRADS:
        assert relerr(got[key], ref[key]) <= 1e-8, key
    for key in KEYS:
        assert relerr(mid[key], xk[key]) <= 1e-10


def test_anchor_loss_through_torch_autograd(P):
    torch = pytest.importorskip("torch")
    g = synth.random_walk_graph(300, n_closures=None, closure_density=1.0, sigma_r=0.02, sigma_t=0.1, seed=4)
    dev = torch.device("cuda:0")
    src = torch.tensor(g.src, dtype=torch.int32, device=dev)
    dst = torch.tensor(g.dst, dtype=torch.int32, device=dev)
    qm = torch.tensor(g.q_meas, dtype=torch.float64, device=dev, requires_grad=True)
    tm = torch.tensor(g.t_meas, dtype=torch.float64, device=dev, requires_grad=True)
    ka = torch.tensor(g.kappa, dtype=torch.float64, device=dev, requires_grad=True)
    om = torch.tensor(g.omega, dtype=torch.float64, device=dev, requires_grad=True)
    prm = P.pradmm_default_params()
    prm.precision = P.PRADMM_FP64
    K = 40
    p, t = P.unrolled_poses(g.n, src, dst, qm, tm, ka, om, iters=K, ckpt_every=10, params=prm)
    from paper_2601_15684_gb300.anchor import anchor_loss as anchor_loss_torch
    L = anchor_loss_torch(p, t, torch.tensor(g.q_gt, device=dev), torch.tensor(g.t_gt, device=dev))
    L.backward()
    q0, t0 = oracle.init_odometry(g)
    st = oracle.init_state(q0, t0)
    x, _, _ = oracle.iterate(g, _oparams(), st, K)
    L_ref, dp, dt = anchor_loss_np(x["p"], x["t"], g.q_gt, g.t_gt)
    assert abs(L.item() - L_ref) <= 1e-8 * L_ref
    ref = oracle.adjoint(g, _oparams(), st, K, dp, dt)
    for key, ten in (("q_meas", qm), ("t_meas", tm), ("kappa", ka), ("omega", om)):
        assert relerr(ten.grad.cpu().numpy(), ref[key]) <= 1e-7, key


def test_adjoint_full_size_walk10k_fp32(P):
    # 10,000-pose walk with ~30,000 edges, 200 unrolled iterations, checkpoint
    # every 20: the reverse-mode workload, against the full oracle reverse pass
    g = synth.workload("walk10k")
    q0, t0 = oracle.init_odometry(g)
    st = oracle.init_state(q0, t0)
    K = 200
    x, _, _ = oracle.iterate(g, _oparams(), st, K)
    _, dp, dt = anchor_loss_np(x["p"], x["t"], g.q_gt, g.t_gt)
    ref = oracle.adjoint(g, _oparams(), st, K, dp, dt)
    with P.Solver(g, precision=1) as S:
        S.init_odometry()
        S.adjoint_record(K, 20)
        got = S.adjoint(dp, dt)
    for key in GRADS:
        assert relerr(got[key], ref[key]) <= 1e-3, (key, relerr(got[key], ref[key]))


def test_reverse_graph_is_reused_and_matches_plain_launches(P):
    # the reverse pass is captured once per tape geometry; a second recording
    # of the same shape from another state reuses the graph
    g = synth.random_graph(180, 500, seed=21)
    st1 = synth.random_state(np.random.default_rng(11), g.n)
    st2 = synth.random_state(np.random.default_rng(12), g.n)
    pb, tb = _cotangent(g.n, 9)
    outs = {}
    for use_graph in (1, 0):
        with P.Solver(g, precision=1, use_graph=use_graph) as S:
            res = []
            for st in (st1, st2, st1):
                S.set_state_full(st)
                S.adjoint_record(17, 5)
                res.append(S.adjoint(pb, tb, x0=True))
            outs[use_graph] = res
    for a, b in zip(outs[1], outs[0]):
        for key in GRADS:
            np.testing.assert_array_equal(a[key], b[key])
        for key in KEYS:
            np.testing.assert_array_equal(a["x0"][key], b["x0"][key])
    for key in GRADS:
        np.testing.assert_array_equal(outs[1][0][key], outs[1][2][key])
        assert not np.array_equal(outs[1][0][key], outs[1][1][key])


def test_automatic_checkpoint_spacing(P):
    # ckpt_every = 0: a small graph's whole tape fits, so every iterate is kept
    # (spacing 1, K + 1 slots of 28 n reals) and the gradients equal those of
    # an explicit spacing bitwise; an explicit spacing is reported as given
    g = synth.random_graph(150, 450, seed=17)
    st = synth.random_state(np.random.default_rng(17), g.n)
    pb, tb = _cotangent(g.n, 4)
    K = 12
    res = {}
    for c in (0, 5):
        with P.Solver(g, precision=1) as S:
            S.set_state_full(st)
            S.adjoint_record(K, c)
            C, nbytes = S.adjoint_tape_info()
            res[c] = S.adjoint(pb, tb, x0=True)
        if c == 0:
            assert C == 1 and nbytes >= (K + 1) * 28 * g.n * 4
        else:
            assert C == 5
    for key in GRADS:
        np.testing.assert_array_equal(res[0][key], res[5][key])
