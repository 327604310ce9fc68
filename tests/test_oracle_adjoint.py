"""Reverse mode of the oracle iteration, pinned by central finite differences.

The oracle's adjoint (a hand-written vector-Jacobian product of every block
of Eq. (3a)-(3f), run backwards through the unrolled iterations) must agree
with FP64 central differences of the forward oracle itself, on measurement
coordinates (q_e, t_e, kappa_e, omega_e) and on the initial state.  Central
differences with h = 1e-6 are accurate to about 1e-9 relative here, so a
dropped term, a wrong sign or a transposed product fails at once.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from oracle.anchor import _conj, _pure, _qmul, anchor_loss
from paper_2601_15684_gb300 import synth

H = 1e-6
KEYS = ("p", "q", "t", "s", "lam", "z")


@pytest.fixture(scope="module")
def case():
    g = synth.random_graph(16, 40, seed=11)
    st = synth.random_state(np.random.default_rng(4), g.n)
    prm = oracle.make_params(beta1=1.0, beta2=1.0, tau=1.5)
    rng = np.random.default_rng(21)
    a, b = rng.normal(size=(g.n, 4)), rng.normal(size=(g.n, 3))
    return g, st, prm, a, b


def _linear(g, prm, st, K, a, b):
    x, _, _ = oracle.iterate(g, prm, st, K)
    return float((a * x["p"]).sum() + (b * x["t"]).sum())


def _fd_measurement(g, key, idx, f):
    vals = []
    for sgn in (1.0, -1.0):
        arr = getattr(g, key).copy()
        arr[idx] += sgn * H
        vals.append(f(dataclasses.replace(g, **{key: arr})))
    return (vals[0] - vals[1]) / (2 * H)


def test_adjoint_matches_central_differences_on_measurements(case):
    g, st, prm, a, b = case
    K = 8
    res = oracle.adjoint(g, prm, st, K, a, b)
    rng = np.random.default_rng(5)
    fd, ad = [], []
    for key, name in (("q_meas", "q_meas"), ("t_meas", "t_meas"), ("kappa", "kappa"), ("omega", "omega")):
        shape = getattr(g, key).shape
        for _ in range(16):  # 64 coordinates in all
            idx = tuple(int(rng.integers(0, s)) for s in shape)
            fd.append(_fd_measurement(g, key, idx, lambda gg: _linear(gg, prm, st, K, a, b)))
            ad.append(res[name][idx])
    fd, ad = np.array(fd), np.array(ad)
    assert np.linalg.norm(fd - ad) <= 1e-6 * np.linalg.norm(ad)
    assert np.abs(fd - ad).max() <= 1e-6 * np.abs(ad).max()
    # and the forward part returns x^K itself
    x, _, _ = oracle.iterate(g, prm, st, K)
    np.testing.assert_array_equal(res["p"], x["p"])
    np.testing.assert_array_equal(res["t"], x["t"])


def test_adjoint_matches_central_differences_on_initial_state(case):
    g, st, prm, a, b = case
    K = 5
    res = oracle.adjoint(g, prm, st, K, a, b)
    rng = np.random.default_rng(8)
    for key in KEYS:
        for _ in range(4):
            idx = (int(rng.integers(0, g.n)), int(rng.integers(0, st[key].shape[1])))
            vals = []
            for sgn in (1.0, -1.0):
                s2 = oracle.copy_state(st)
                s2[key][idx] += sgn * H
                vals.append(_linear(g, prm, s2, K, a, b))
            fd = (vals[0] - vals[1]) / (2 * H)
            ad = res["x0"][key][idx]
            assert abs(fd - ad) <= 1e-6 * max(1.0, abs(ad)), (key, idx, fd, ad)


def test_anchor_loss_gradient_by_differences():
    rng = np.random.default_rng(2)
    n = 7
    p = rng.normal(size=(n, 4))
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    t = rng.normal(size=(n, 3)) * 3
    q_gt = rng.normal(size=(n, 4))
    q_gt /= np.linalg.norm(q_gt, axis=1, keepdims=True)
    t_gt = t + rng.normal(size=(n, 3)) * 0.3
    L, dp, dt = anchor_loss(p, t, q_gt, t_gt)
    for arr, grad in ((p, dp), (t, dt)):
        for idx in np.ndindex(arr.shape):
            if arr is p and idx[0] > 0:
                assert grad[idx] == 0.0
                continue
            a1, a2 = arr.copy(), arr.copy()
            a1[idx] += H
            a2[idx] -= H
            f1 = anchor_loss(a1, t, q_gt, t_gt)[0] if arr is p else anchor_loss(p, a1, q_gt, t_gt)[0]
            f2 = anchor_loss(a2, t, q_gt, t_gt)[0] if arr is p else anchor_loss(p, a2, q_gt, t_gt)[0]
            assert abs((f1 - f2) / (2 * H) - grad[idx]) <= 1e-6 * max(1.0, abs(grad[idx]))
    # zero at the ground truth moved by any global rigid motion (gauge of Eq. (1))
    g = np.array([np.cos(0.3), 0.0, np.sin(0.3), 0.0])
    moved = _qmul(_qmul(g[None], _pure(t_gt)), _conj(g)[None])[:, 1:] + np.array([5.0, -2.0, 1.0])
    assert anchor_loss(_qmul(g[None], q_gt), moved, q_gt, t_gt)[0] < 1e-20


def test_anchor_loss_through_iterations_by_differences():
    g = synth.random_walk_graph(40, n_closures=None, closure_density=1.0, sigma_r=0.02, sigma_t=0.1, seed=3)
    q0, t0 = oracle.init_odometry(g)
    st = oracle.init_state(q0, t0)
    prm = oracle.make_params(beta1=1.0, beta2=1.0, tau=1.5)
    K = 12
    x, _, _ = oracle.iterate(g, prm, st, K)
    _, dp, dt = anchor_loss(x["p"], x["t"], g.q_gt, g.t_gt)
    res = oracle.adjoint(g, prm, st, K, dp, dt)

    def f(gg):
        xx, _, _ = oracle.iterate(gg, prm, st, K)
        return anchor_loss(xx["p"], xx["t"], g.q_gt, g.t_gt)[0]

    rng = np.random.default_rng(1)
    for key in ("q_meas", "t_meas", "kappa", "omega"):
        for _ in range(3):
            idx = tuple(int(rng.integers(0, s)) for s in getattr(g, key).shape)
            fd = _fd_measurement(g, key, idx, f)
            assert abs(fd - res[key][idx]) <= 1e-6 * max(1.0, np.abs(res[key]).max()), (key, idx)


def test_adjoint_of_zero_iterations_is_the_cotangent(case):
    g, st, prm, a, b = case
    res = oracle.adjoint(g, prm, st, 0, a, b)
    for key in ("q_meas", "t_meas", "kappa", "omega"):
        assert not res[key].any()
    np.testing.assert_array_equal(res["x0"]["p"], a)
    np.testing.assert_array_equal(res["x0"]["t"], b)
    for key in ("q", "s", "lam", "z"):
        assert not res["x0"][key].any()


# ---- the inertial iteration (reading R27) ----------------------------------------

def _linear_inertial(g, prm, st, K, theta, a, b):
    x, _, _, _ = oracle.iterate_inertial(g, prm, st, theta, K)
    return float((a * x["p"]).sum() + (b * x["t"]).sum())


@pytest.fixture(scope="module")
def icase():
    # proximal weights large enough that the anchors carry weight
    g = synth.random_graph(14, 36, seed=12)
    st = synth.random_state(np.random.default_rng(6), g.n)
    prm = oracle.make_params(beta1=1.0, beta2=1.0, tau=1.5, gamma=(1.0, 0.6, 0.5, 0.7))
    rng = np.random.default_rng(22)
    a, b = rng.normal(size=(g.n, 4)), rng.normal(size=(g.n, 3))
    return g, st, prm, a, b


def test_inertial_adjoint_with_zero_theta_is_the_plain_adjoint(icase):
    g, st, prm, a, b = icase
    r0 = oracle.adjoint(g, prm, st, 6, a, b)
    r1 = oracle.adjoint_inertial(g, prm, st, 6, 0.0, a, b)
    for key in ("p", "t", "q_meas", "t_meas", "kappa", "omega"):
        np.testing.assert_array_equal(r0[key], r1[key])
    for key in KEYS:
        np.testing.assert_array_equal(r0["x0"][key], r1["x0"][key])


@pytest.mark.parametrize("theta", [0.4, 0.8])
def test_inertial_adjoint_matches_central_differences_on_measurements(icase, theta):
    g, st, prm, a, b = icase
    K = 7
    res = oracle.adjoint_inertial(g, prm, st, K, theta, a, b)
    rng = np.random.default_rng(15)
    fd, ad = [], []
    for key in ("q_meas", "t_meas", "kappa", "omega"):
        shape = getattr(g, key).shape
        for _ in range(12):
            idx = tuple(int(rng.integers(0, s)) for s in shape)
            fd.append(_fd_measurement(g, key, idx, lambda gg: _linear_inertial(gg, prm, st, K, theta, a, b)))
            ad.append(res[key][idx])
    fd, ad = np.array(fd), np.array(ad)
    assert np.linalg.norm(fd - ad) <= 1e-6 * np.linalg.norm(ad)
    assert np.abs(fd - ad).max() <= 1e-6 * np.abs(ad).max()
    x, _, _, _ = oracle.iterate_inertial(g, prm, st, theta, K)
    np.testing.assert_array_equal(res["p"], x["p"])
    np.testing.assert_array_equal(res["t"], x["t"])


def test_inertial_adjoint_matches_central_differences_on_initial_state(icase):
    # x^0 enters twice (as x^0 and as x^{-1}); the adjoint holds both shares
    g, st, prm, a, b = icase
    K, theta = 5, 0.6
    res = oracle.adjoint_inertial(g, prm, st, K, theta, a, b)
    rng = np.random.default_rng(18)
    for key in KEYS:
        for _ in range(4):
            idx = (int(rng.integers(0, g.n)), int(rng.integers(0, st[key].shape[1])))
            vals = []
            for sgn in (1.0, -1.0):
                s2 = oracle.copy_state(st)
                s2[key][idx] += sgn * H
                vals.append(_linear_inertial(g, prm, s2, K, theta, a, b))
            fd = (vals[0] - vals[1]) / (2 * H)
            ad = res["x0"][key][idx]
            assert abs(fd - ad) <= 1e-6 * max(1.0, abs(ad)), (key, idx, fd, ad)
