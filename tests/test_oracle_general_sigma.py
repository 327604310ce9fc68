"""Pins of the general-Sigma oracle (Lemma 1, Algorithm 2, Appendix B/C).

- the sphere-constrained quadratic (Lemma 1) solved by Algorithm 2 against
  brute force on S^3, including the hard case, and its optimality conditions;
- Sigma_1 = c1 I, Sigma_2 = c2 I reduce to the pinned scalar C oracle with the
  weights scaled;
- every block of one iteration minimises its exact subproblem of the
  augmented Lagrangian (evaluated here from its definition) for random SPD
  Sigma_1, Sigma_2: p over sampled points of S^3 and with zero Riemannian
  gradient, q, t, s with zero gradient;
- the noise-free ground truth is a fixed point for any Sigma.
"""
import numpy as np
import pytest

import oracle
from oracle import general_sigma as gs
from paper_2601_15684_gb300 import synth

PARAMS = (1.0, 1.0, 1.5, (1.0, 1e-3, 1e-3, 1e-3))


def _spd(rng, k, cond=5.0):
    Q, _ = np.linalg.qr(rng.normal(size=(k, k)))
    return Q @ np.diag(np.exp(rng.uniform(0, np.log(cond), k))) @ Q.T


def _brute_sphere(A, b, rng, samples=200000):
    f = lambda x: 0.5 * np.einsum("...i,ij,...j->...", x, A, x) + x @ b
    X = rng.normal(size=(samples, 4))
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    best = X[np.argsort(f(X))[:8]]
    out = []
    for x in best:  # Riemannian gradient descent polish
        for _ in range(3000):
            gr = A @ x + b
            gr -= (gr @ x) * x
            x = x - 0.05 * gr / max(1.0, np.abs(A).max())
            x /= np.linalg.norm(x)
        out.append(x)
    vals = [f(x) for x in out]
    return out[int(np.argmin(vals))], min(vals)


@pytest.mark.parametrize("seed", range(6))
def test_trs_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    B = rng.normal(size=(4, 4))
    A = B + B.T
    b = rng.normal(size=4) * rng.uniform(0.1, 3.0)
    x, lam, hard = gs.trs_sphere(A, b)
    f = lambda y: 0.5 * y @ A @ y + b @ y
    _, fb = _brute_sphere(A, b, rng)
    # lambda* comes from an 8x8 nonsymmetric eigenproblem: |x| = 1 to ~1e-12
    assert abs(np.linalg.norm(x) - 1) < 1e-10
    assert f(x) <= fb + 1e-10
    assert np.linalg.norm((A + lam * np.eye(4)) @ x + b) < 1e-9
    assert np.linalg.eigvalsh(A + lam * np.eye(4)).min() > -1e-9
    assert not hard


def test_trs_hard_case():
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.normal(size=(4, 4)))
    A = Q @ np.diag([-2.0, 1.0, 3.0, 4.0]) @ Q.T
    # b with no component on the eigenvector of -2 and small enough that
    # |-(A + 2 I)^+ b| < 1: the minimiser needs the null-space component
    b = Q @ np.array([0.0, 0.5, 0.8, -0.3])
    x, lam, hard = gs.trs_sphere(A, b)
    assert hard and abs(lam - 2.0) < 1e-9
    f = lambda y: 0.5 * y @ A @ y + b @ y
    _, fb = _brute_sphere(A, b, rng)
    assert abs(np.linalg.norm(x) - 1) < 1e-10 and f(x) <= fb + 1e-10
    assert np.linalg.norm((A + lam * np.eye(4)) @ x + b) < 1e-9
    # the sign of the null-space component follows the previous iterate
    v = Q[:, 0]
    x_plus, _, _ = gs.trs_sphere(A, b, x_prev=v)
    x_minus, _, _ = gs.trs_sphere(A, b, x_prev=-v)
    assert x_plus @ v > 0 > x_minus @ v


def test_trs_scalar_matrix_is_the_closed_form():
    rng = np.random.default_rng(5)
    for _ in range(10):
        b = rng.normal(size=4)
        x, lam, _ = gs.trs_sphere(3.7 * np.eye(4), b)
        np.testing.assert_allclose(x, -b / np.linalg.norm(b), atol=1e-12)
        assert abs(lam - (np.linalg.norm(b) - 3.7)) < 1e-10


@pytest.mark.parametrize("c1,c2", [(1.0, 1.0), (2.5, 0.4)])
def test_scalar_sigma_reduces_to_the_c_oracle(c1, c2):
    g = synth.random_graph(12, 30, seed=2)
    st = synth.random_state(np.random.default_rng(1), g.n)
    x, e, hard = gs.iterate(g, PARAMS, c1 * np.eye(4), c2 * np.eye(4), st)
    import dataclasses
    g2 = dataclasses.replace(g, omega=g.omega * c1, kappa=g.kappa * c2)
    ref, res, _ = oracle.iterate(g2, oracle.make_params(beta1=1.0, beta2=1.0, tau=1.5), st, 1)
    for key in ("p", "q", "t", "s", "lam", "z"):
        np.testing.assert_allclose(x[key], ref[key], rtol=1e-11, atol=1e-11)
    assert abs(e - res[0]) <= 1e-11 * max(res[0], 1.0)
    assert hard == 0


def _num_grad(f, x, h=1e-6):
    gr = np.zeros_like(x)
    for idx in np.ndindex(x.shape):
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        gr[idx] = (f(xp) - f(xm)) / (2 * h)
    return gr


@pytest.mark.parametrize("seed", [0, 1])
def test_every_block_minimises_its_subproblem(seed):
    rng = np.random.default_rng(seed)
    g = synth.random_graph(6, 14, seed=10 + seed)
    st = synth.random_state(rng, g.n)
    S1, S2 = _spd(rng, 4), _spd(rng, 4)
    b1, b2, tau, (g1, g2, g3, g4) = PARAMS
    new, _, _ = gs.iterate(g, PARAMS, S1, S2, st)
    L = lambda s: gs.lagrangian(g, PARAMS, S1, S2, s)

    def with_(base, **kw):
        d = {k: v.copy() for k, v in base.items()}
        d.update(kw)
        return d

    # p-block: per vertex on S^3 (the Lagrangian separates over p_i)
    for i in range(g.n):
        def fp(x):
            p = new["p"].copy()
            p[i] = x
            return L(with_(st, p=p)) + 0.5 * g1 * np.sum((x - st["p"][i]) ** 2)
        x0 = new["p"][i]
        f0 = fp(x0)
        X = rng.normal(size=(2000, 4))
        X /= np.linalg.norm(X, axis=1, keepdims=True)
        assert min(fp(x) for x in X) >= f0 - 1e-9
        gr = _num_grad(fp, x0)
        gr -= (gr @ x0) * x0
        assert np.linalg.norm(gr) < 1e-5
    # q, t, s blocks: zero gradient of their subproblems
    fq = lambda q: L(with_(st, p=new["p"], q=q)) + 0.5 * g2 * np.sum((q - st["q"]) ** 2)
    assert np.abs(_num_grad(fq, new["q"])).max() < 1e-5
    ft = lambda t: L(with_(st, p=new["p"], q=new["q"], t=t)) + 0.5 * g3 * np.sum((t - st["t"]) ** 2)
    assert np.abs(_num_grad(ft, new["t"])).max() < 1e-5
    fs = lambda s: (L(with_(st, p=new["p"], q=new["q"], t=new["t"], s=s))
                    + 0.5 * g4 * np.sum((s - st["s"]) ** 2))
    assert np.abs(_num_grad(fs, new["s"])).max() < 1e-5


def test_noise_free_truth_is_a_fixed_point_for_any_sigma():
    rng = np.random.default_rng(4)
    g = synth.random_walk_graph(20, n_closures=15, sigma_r=0.0, sigma_t=0.0, seed=2)
    S1, S2 = _spd(rng, 4), _spd(rng, 4)
    st = oracle.init_state(g.q_gt, g.t_gt)
    x, e, _ = gs.iterate(g, PARAMS, S1, S2, st)
    assert e < 1e-24
    for key in ("p", "q"):
        np.testing.assert_allclose(x[key], g.q_gt, atol=1e-12)
    for key in ("t", "s"):
        np.testing.assert_allclose(x[key], g.t_gt, atol=1e-12)
    assert gs.objective(g, S1, S2, g.q_gt, g.t_gt) < 1e-24


def test_p_system_matches_iterate():
    rng = np.random.default_rng(9)
    g = synth.random_graph(8, 20, seed=4)
    st = synth.random_state(rng, g.n)
    S1, S2 = _spd(rng, 4), _spd(rng, 4)
    new, _, _ = gs.iterate(g, PARAMS, S1, S2, st)
    for i in range(g.n):
        A1, b1 = gs.p_system(g, PARAMS, S1, S2, st, i)
        x, _, _ = gs.trs_sphere(A1, b1, st["p"][i])
        np.testing.assert_allclose(x, new["p"][i], atol=1e-12)


# ---- inertial variant (reading R27) -------------------------------------------

def test_inertial_zero_theta_is_plain():
    rng = np.random.default_rng(21)
    g = synth.random_graph(9, 24, seed=6)
    st = synth.random_state(rng, g.n)
    prev = synth.random_state(rng, g.n)
    S1, S2 = _spd(rng, 4), _spd(rng, 4)
    a, e_a, h_a = gs.iterate(g, PARAMS, S1, S2, st)
    b, pv, e_b, h_b = gs.iterate_inertial(g, PARAMS, S1, S2, st, 0.0, prev)
    for key in a:
        np.testing.assert_array_equal(a[key], b[key])
    assert e_a == e_b and h_a == h_b
    for key in ("p", "q", "t", "s"):
        np.testing.assert_array_equal(pv[key], st[key])


@pytest.mark.parametrize("theta", [0.3, 0.8])
def test_inertial_identity_sigma_reduces_to_the_c_oracle(theta):
    # Sigma = I is the scalar model: two inertial iterations of this module
    # against the C oracle's inertial iteration (pinned on its own)
    rng = np.random.default_rng(22)
    g = synth.random_graph(14, 40, seed=7)
    st = synth.random_state(rng, g.n)
    prev = {k: v for k, v in synth.random_state(rng, g.n).items() if k in ("p", "q", "t", "s")}
    x, pv = st, prev
    for _ in range(2):
        x, pv, e, hard = gs.iterate_inertial(g, PARAMS, np.eye(4), np.eye(4), x, theta, pv)
    prm = oracle.make_params(beta1=PARAMS[0], beta2=PARAMS[1], tau=PARAMS[2], gamma=PARAMS[3])
    ref, ref_pv, res, _ = oracle.iterate_inertial(g, prm, st, theta, 2, prev)
    for key in ("p", "q", "t", "s", "lam", "z"):
        np.testing.assert_allclose(x[key], ref[key], rtol=1e-11, atol=1e-11)
    for key in ("p", "q", "t", "s"):
        np.testing.assert_allclose(pv[key], ref_pv[key], rtol=1e-11, atol=1e-11)
    assert abs(e - res[0]) <= 1e-11 * max(res[0], 1.0)
    assert hard == 0


def test_inertial_blocks_minimise_around_extrapolated_anchors():
    # each block minimises its subproblem of L_beta plus 1/2 gamma |x - a|^2,
    # the anchor a formed here from x^k and x^{k-1}
    rng = np.random.default_rng(23)
    g = synth.random_graph(6, 14, seed=12)
    st = synth.random_state(rng, g.n)
    prev = synth.random_state(rng, g.n)
    S1, S2 = _spd(rng, 4), _spd(rng, 4)
    theta = 0.6
    prm = (1.0, 1.0, 1.5, (1.0, 0.7, 0.4, 0.9))  # proximal weights large enough to see the anchors
    _, _, _, (g1, g2, g3, g4) = prm
    new, _, _, _ = gs.iterate_inertial(g, prm, S1, S2, st, theta, prev)
    a = {k: st[k] + theta * (st[k] - prev[k]) for k in ("p", "q", "t", "s")}
    L = lambda s: gs.lagrangian(g, prm, S1, S2, s)

    def with_(base, **kw):
        d = {k: v.copy() for k, v in base.items()}
        d.update(kw)
        return d

    for i in range(g.n):
        def fp(x):
            p = new["p"].copy()
            p[i] = x
            return L(with_(st, p=p)) + 0.5 * g1 * np.sum((x - a["p"][i]) ** 2)
        x0 = new["p"][i]
        f0 = fp(x0)
        X = rng.normal(size=(2000, 4))
        X /= np.linalg.norm(X, axis=1, keepdims=True)
        assert min(fp(x) for x in X) >= f0 - 1e-9
        gr = _num_grad(fp, x0)
        gr -= (gr @ x0) * x0
        assert np.linalg.norm(gr) < 1e-5
    fq = lambda q: L(with_(st, p=new["p"], q=q)) + 0.5 * g2 * np.sum((q - a["q"]) ** 2)
    assert np.abs(_num_grad(fq, new["q"])).max() < 1e-5
    ft = lambda t: L(with_(st, p=new["p"], q=new["q"], t=t)) + 0.5 * g3 * np.sum((t - a["t"]) ** 2)
    assert np.abs(_num_grad(ft, new["t"])).max() < 1e-5
    fs = lambda s: (L(with_(st, p=new["p"], q=new["q"], t=new["t"], s=s))
                    + 0.5 * g4 * np.sum((s - a["s"]) ** 2))
    assert np.abs(_num_grad(fs, new["s"])).max() < 1e-5


def test_inertial_noise_free_truth_is_a_fixed_point_for_any_sigma():
    rng = np.random.default_rng(24)
    g = synth.random_walk_graph(20, n_closures=15, sigma_r=0.0, sigma_t=0.0, seed=3)
    S1, S2 = _spd(rng, 4), _spd(rng, 4)
    st = oracle.init_state(g.q_gt, g.t_gt)
    x, pv = st, None
    for _ in range(3):
        x, pv, e, _ = gs.iterate_inertial(g, PARAMS, S1, S2, x, 0.5, pv)
    assert e < 1e-24
    for key in ("p", "q"):
        np.testing.assert_allclose(x[key], g.q_gt, atol=1e-12)
    for key in ("t", "s"):
        np.testing.assert_allclose(x[key], g.t_gt, atol=1e-12)
