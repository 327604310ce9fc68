"""Pins of the oracle's PRADMM iteration against what the paper fixes.

- T3  product forms == literal matrix forms of Appendix B (two statements).
- T4  every block update minimises its exact subproblem (Eq. (3a)-(3d)) --
      brute force on S^3 for p, zero gradient + positive curvature for q, t, s;
      the augmented Lagrangian is evaluated here from its definition
      (Section 3.2 with the split model (2)), independently of the oracle.
- T5  noise-free ground truth with zero multipliers is a fixed point.
- T6  noise-free recovery from a perturbed start, F -> 0 up to a gauge.
- T7  one step commutes with a global SE(3) motion (F is gauge invariant).
- T8  convergence: e^k -> 0, p - q -> 0, t - s -> 0, F decreases (Thm 1).
- T9  the augmented Lagrangian is non-increasing after a burn-in.
- T10 the Riemannian KKT residual (optimality lemma, Appendix D) shrinks.
- T12 |u_i| = 0 keeps p_i^k (reading R11).
- odometry initialisation recovers noise-free ground truth.
"""
import numpy as np
import pytest

import oracle
from oracle import matrix_form as mf
from paper_2601_15684_gb300 import synth

BETA1, BETA2, TAU, GAMMA = 3.0, 5.0, 1.3, (0.7, 0.01, 0.02, 0.03)


def P():
    return oracle.make_params(beta1=BETA1, beta2=BETA2, tau=TAU, gamma=GAMMA)


# ---- an independent evaluation of L_beta + Q_s from the definitions ------

def _qm(a, b):
    # scalar-first Hamilton product, written from p q = [p0 q0 - p.q, p0 q + q0 p + p x q]
    a0, av = a[..., :1], a[..., 1:]
    b0, bv = b[..., :1], b[..., 1:]
    return np.concatenate([a0 * b0 - np.sum(av * bv, -1, keepdims=True),
                           a0 * bv + b0 * av + np.cross(av, bv)], -1)


def _cj(a):
    return a * np.array([1.0, -1, -1, -1])


def _pure(t):
    return np.concatenate([np.zeros(t.shape[:-1] + (1,)), t], -1)


def lagrangian(g, st, beta1, beta2):
    i, j = g.src, g.dst
    p, q, t, s, lam, z = (st[k] for k in ("p", "q", "t", "s", "lam", "z"))
    r1 = _pure(t[j]) - _pure(s[i]) - _qm(_qm(q[i], _pure(g.t_meas)), _cj(p[i]))
    r2 = _qm(_qm(_cj(p[j]), q[i]), g.q_meas) - np.array([1.0, 0, 0, 0])
    f = np.sum(g.omega * np.sum(r1 * r1, -1))
    gg = np.sum(g.kappa * np.sum(r2 * r2, -1))
    L = f + gg
    L += np.sum(-np.sum(lam * (p - q), -1) + 0.5 * beta1 * np.sum((p - q) ** 2, -1))
    L += np.sum(-np.sum(z * (t - s), -1) + 0.5 * beta2 * np.sum((t - s) ** 2, -1))
    return L


def _graphs():
    yield synth.random_graph(6, 14, seed=10, isolated=1)
    yield synth.random_graph(5, 9, seed=11)
    yield synth.random_walk_graph(6, n_closures=4, seed=12)


def _state(g, seed):
    return synth.random_state(np.random.default_rng(seed), g.n)


# ---- T3 ---------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_product_form_equals_matrix_form(seed):
    g = synth.random_graph(15, 60, seed=100 + seed, isolated=2)
    st = _state(g, seed)
    a, res, _ = oracle.iterate(g, P(), st)
    b, e, dev = mf.iterate(g, BETA1, BETA2, TAU, GAMMA, st)
    for k in a:
        scale = max(1.0, np.abs(b[k]).max())
        assert np.abs(a[k] - b[k]).max() <= 1e-13 * scale, k
    assert abs(res[0] - e) <= 1e-12 * max(1.0, e)
    # Lemma MW(c): with scalar Sigma the matrices A_1 and A_2 are scalar (Section 3.3)
    assert dev["A1"] < 1e-12 and dev["A2"] < 1e-12


def test_oracle_lagrangian_matches_definition():
    for g in _graphs():
        st = _state(g, 5)
        assert abs(oracle.lagrangian(g, P(), st) - lagrangian(g, st, BETA1, BETA2)) < 1e-11


def _edge_terms(g, q, t):
    """Per-edge squared residuals of Eq. (1), written out here from the
    problem statement: translation |t~_j - t~_i - q_i t~_ij q_i^*|^2 and
    rotation |q_j^* q_i q_ij - 1|^2."""
    i, j = g.src, g.dst
    r1 = _pure(t[j]) - _pure(t[i]) - _qm(_qm(q[i], _pure(g.t_meas)), _cj(q[i]))
    r2 = _qm(_qm(_cj(q[j]), q[i]), g.q_meas) - np.array([1.0, 0, 0, 0])
    return np.sum(r1 * r1, -1), np.sum(r2 * r2, -1)


def test_oracle_objective_matches_definition_with_edge_weights():
    # Eq. (1) with per-edge weights omega_e (translation) and kappa_e
    # (rotation), drawn independently so that swapping them, dropping one,
    # or using the head's weight instead of the edge's changes F
    rng = np.random.default_rng(21)
    for g in _graphs():
        g = synth.PoseGraph(n=g.n, src=g.src, dst=g.dst, q_meas=g.q_meas, t_meas=g.t_meas,
                            kappa=rng.uniform(0.1, 3.0, g.m), omega=rng.uniform(0.1, 3.0, g.m))
        st = _state(g, 6)
        q, t = st["q"], st["t"]
        ft, fr = _edge_terms(g, q, t)
        F = oracle.objective(g, q, t)
        F_def = float(np.sum(g.omega * ft) + np.sum(g.kappa * fr))
        assert abs(F - F_def) <= 1e-12 * F_def, (F, F_def)
        # F is the split model's L_beta at p = q, s = t with zero multipliers
        x = dict(st, p=q, s=t, lam=np.zeros_like(st["lam"]), z=np.zeros_like(st["z"]))
        assert abs(F - lagrangian(g, x, BETA1, BETA2)) <= 1e-12 * F_def
        # each weight reaches its own term only
        only_t = synth.PoseGraph(n=g.n, src=g.src, dst=g.dst, q_meas=g.q_meas, t_meas=g.t_meas,
                                 kappa=np.zeros(g.m), omega=g.omega)
        only_r = synth.PoseGraph(n=g.n, src=g.src, dst=g.dst, q_meas=g.q_meas, t_meas=g.t_meas,
                                 kappa=g.kappa, omega=np.zeros(g.m))
        assert abs(oracle.objective(only_t, q, t) - np.sum(g.omega * ft)) <= 1e-12 * F_def
        assert abs(oracle.objective(only_r, q, t) - np.sum(g.kappa * fr)) <= 1e-12 * F_def
        # one edge's weight moves F by that edge's own term
        e = g.m // 2
        w2 = g.omega.copy()
        w2[e] += 1.0
        bumped = synth.PoseGraph(n=g.n, src=g.src, dst=g.dst, q_meas=g.q_meas, t_meas=g.t_meas,
                                 kappa=g.kappa, omega=w2)
        assert abs(oracle.objective(bumped, q, t) - F - ft[e]) <= 1e-12 * F_def


# ---- T4 brute force ---------------------------------------------------------

def _blocks(g, st, new):
    """States at which each block is solved in Eq. (3a)-(3d)."""
    x_p = dict(st)
    x_q = dict(st, p=new["p"])
    x_t = dict(st, p=new["p"], q=new["q"])
    x_s = dict(st, p=new["p"], q=new["q"], t=new["t"])
    return x_p, x_q, x_t, x_s


def _obj(g, base, key, i, v, anchor, gam):
    st = dict(base)
    arr = base[key].copy()
    arr[i] = v
    st[key] = arr
    return lagrangian(g, st, BETA1, BETA2) + 0.5 * gam * np.sum((v - anchor) ** 2)


@pytest.mark.parametrize("gi", [0, 1, 2])
def test_p_block_is_sphere_minimiser(gi):
    g = list(_graphs())[gi]
    st = _state(g, 20 + gi)
    new, _, _ = oracle.iterate(g, P(), st)
    x_p = _blocks(g, st, new)[0]
    rng = np.random.default_rng(7)
    cloud = rng.standard_normal((20000, 4))
    cloud /= np.linalg.norm(cloud, axis=1, keepdims=True)
    for i in range(g.n):
        anchor = st["p"][i]
        f = lambda v: _obj(g, x_p, "p", i, v, anchor, GAMMA[0])
        p_star = new["p"][i]
        assert abs(np.linalg.norm(p_star) - 1) < 1e-14
        f_star = f(p_star)
        # the closed form beats every sampled point of S^3
        vals = np.array([f(v) for v in cloud[::10]])
        assert f_star <= vals.min() + 1e-12
        # and the Riemannian gradient (I - p p^T) grad f vanishes (finite differences)
        h = 1e-5
        grad = np.array([(f(p_star + h * e) - f(p_star - h * e)) / (2 * h) for e in np.eye(4)])
        rg = grad - p_star * (p_star @ grad)
        assert np.linalg.norm(rg) < 1e-6 * max(1.0, np.linalg.norm(grad))
        # the stationary point is the minimiser, not the antipodal maximiser
        assert f_star < f(-p_star)


@pytest.mark.parametrize("gi", [0, 1, 2])
def test_q_t_s_blocks_zero_gradient(gi):
    g = list(_graphs())[gi]
    st = _state(g, 30 + gi)
    new, _, _ = oracle.iterate(g, P(), st)
    _, x_q, x_t, x_s = _blocks(g, st, new)
    for key, base, gam, dim in (("q", x_q, GAMMA[1], 4), ("t", x_t, GAMMA[2], 3), ("s", x_s, GAMMA[3], 3)):
        for i in range(g.n):
            anchor = st[key][i]
            v = new[key][i]
            f = lambda w: _obj(g, base, key, i, w, anchor, gam)
            h = 1e-3  # the objective is quadratic in each block: central differences are exact
            E = np.eye(dim)
            grad = np.array([(f(v + h * e) - f(v - h * e)) / (2 * h) for e in E])
            assert np.linalg.norm(grad) < 1e-7 * max(1.0, abs(f(v))), (key, i, grad)
            H = np.array([[(f(v + h * a + h * b) - f(v + h * a - h * b) - f(v - h * a + h * b)
                            + f(v - h * a - h * b)) / (4 * h * h) for b in E] for a in E])
            assert np.linalg.eigvalsh(0.5 * (H + H.T)).min() > 0


# ---- T5, T6 -----------------------------------------------------------------

def _noise_free_graphs():
    yield synth.random_walk_graph(64, n_closures=60, sigma_r=0.0, sigma_t=0.0, seed=7)
    yield synth.helix_graph(n=450, sigma_r=0.0, sigma_t=0.0)
    yield synth.random_graph(30, 90, seed=8, sigma_r=0.0, sigma_t=0.0)


@pytest.mark.parametrize("gi", [0, 1, 2])
def test_noise_free_truth_is_fixed_point(gi):
    g = list(_noise_free_graphs())[gi]
    st = oracle.init_state(g.q_gt, g.t_gt)
    new, res, _ = oracle.iterate(g, P(), st)
    for k in st:
        assert np.abs(new[k] - st[k]).max() < 1e-12, k
    assert res[0] < 1e-20
    assert oracle.objective(g, g.q_gt, g.t_gt) < 1e-24 * g.m + 1e-24


def test_noise_free_recovery_up_to_gauge():
    g = synth.random_walk_graph(40, n_closures=40, sigma_r=0.0, sigma_t=0.0, seed=11)
    rng = np.random.default_rng(5)
    q0 = synth._qmul(g.q_gt, synth.axis_angle_noise(rng, g.n, 0.1))
    t0 = g.t_gt + 0.1 * rng.standard_normal((g.n, 3))
    prm = oracle.make_params(beta1=1.0, beta2=1.0, tau=1.5)
    st, k, e, _ = oracle.solve(g, prm, oracle.init_state(q0, t0), 4000, 0.0)
    F = oracle.objective(g, st["p"], st["t"])
    assert F < 1e-12 * g.m
    # align the gauge on pose 0: g = p_0 q_gt0^*, then compare all poses
    gq = synth._qmul(st["p"][0], synth._qconj(g.q_gt[0]))
    q_al = synth._qmul(np.broadcast_to(gq, g.q_gt.shape), g.q_gt)
    sign = np.sign(np.sum(q_al * st["p"], axis=1, keepdims=True))
    assert np.abs(sign * q_al - st["p"]).max() < 1e-5
    t_al = synth._rotate(np.broadcast_to(gq, (g.n, 4)), g.t_gt - g.t_gt[0]) + st["t"][0]
    assert np.abs(t_al - st["t"]).max() < 1e-5


# ---- T7 ---------------------------------------------------------------------

def test_step_commutes_with_global_se3():
    g = synth.random_graph(20, 70, seed=13, isolated=1)
    st = _state(g, 14)
    rng = np.random.default_rng(15)
    gq = synth.random_unit_quaternions(rng, 1)[0]
    d = rng.standard_normal(3)

    def move(x):
        G = np.broadcast_to(gq, x["p"].shape)
        R = lambda v: synth._rotate(np.broadcast_to(gq, v.shape[:-1] + (4,)), v)
        return {"p": synth._qmul(G, x["p"]), "q": synth._qmul(G, x["q"]), "lam": synth._qmul(G, x["lam"]),
                "t": R(x["t"]) + d, "s": R(x["s"]) + d, "z": R(x["z"])}

    a, ra, _ = oracle.iterate(g, P(), move(st))
    b, rb, _ = oracle.iterate(g, P(), st)
    mb = move(b)
    for k in a:
        assert np.abs(a[k] - mb[k]).max() < 1e-11, k
    assert abs(ra[0] - rb[0]) < 1e-10 * max(1, rb[0])
    assert abs(oracle.objective(g, a["p"], a["t"]) - oracle.objective(g, b["p"], b["t"])) < 1e-9


# ---- T8, T9, T10 --------------------------------------------------------------

def _kkt_residual(g, st, beta1, beta2):
    """Riemannian KKT residual of the optimality lemma (Appendix D) for the
    split model at (x, lambda): projected gradient of f + g - <lambda, A x>
    in p, plain gradients in q, t, s, and the feasibility p - q, t - s;
    derivatives by central differences of L_beta with the penalty removed."""
    def L0(x):
        return lagrangian(g, x, 0.0, 0.0)
    tot = 0.0
    h = 1e-6
    for key in ("p", "q", "t", "s"):
        arr = st[key]
        gr = np.zeros_like(arr)
        for i in range(arr.shape[0]):
            for c in range(arr.shape[1]):
                xp = dict(st); ap = arr.copy(); ap[i, c] += h; xp[key] = ap
                xm = dict(st); am = arr.copy(); am[i, c] -= h; xm[key] = am
                gr[i, c] = (L0(xp) - L0(xm)) / (2 * h)
        if key == "p":
            gr = gr - arr * np.sum(arr * gr, axis=1, keepdims=True)
        tot += np.sum(gr ** 2)
    tot += np.sum((st["p"] - st["q"]) ** 2) + np.sum((st["t"] - st["s"]) ** 2)
    return np.sqrt(tot)


def test_convergence_walk128():
    g = synth.workload("walk128")
    q0, t0 = oracle.init_odometry(g)
    prm = oracle.make_params(beta1=1.0, beta2=1.0, tau=1.5)
    st0 = oracle.init_state(q0, t0)
    st, k, e, trace = oracle.solve(g, prm, st0, 500, 0.0)
    assert trace[-1] < 1e-4 * trace[0]
    # e^k -> 0 (Thm 1(ii)); a monotone envelope over windows of 50 iterations
    w = trace[: 500].reshape(10, 50).max(axis=1)
    assert np.all(np.diff(w[2:]) < 0)
    assert np.abs(st["p"] - st["q"]).max() < 1e-3
    assert np.abs(st["t"] - st["s"]).max() < 1e-3
    F0 = oracle.objective(g, q0, t0)
    F1 = oracle.objective(g, st["p"], st["t"])
    assert F1 < 0.5 * F0
    # T9: the augmented Lagrangian decreases after a burn-in of 20 iterations
    x = st0
    L = []
    for it in range(120):
        x, _, _ = oracle.iterate(g, prm, x)
        L.append(oracle.lagrangian(g, prm, x))
    assert np.all(np.diff(L[20:]) <= 1e-12)


def test_convergence_helix_and_kkt():
    g = synth.helix_graph(n=600)
    q0, t0 = oracle.init_odometry(g)
    prm = oracle.make_params(beta1=1.0, beta2=1.0, tau=1.5)
    st0 = oracle.init_state(q0, t0)
    s1, _, e1, tr = oracle.solve(g, prm, st0, 300, 0.0)
    assert tr[-1] < 1e-3 * tr[0]
    assert oracle.objective(g, s1["p"], s1["t"]) < oracle.objective(g, q0, t0)
    small = synth.random_walk_graph(24, n_closures=20, seed=21)
    q0, t0 = oracle.init_odometry(small)
    x0 = oracle.init_state(q0, t0)
    k_early = _kkt_residual(small, oracle.solve(small, prm, x0, 20, 0.0)[0], 1.0, 1.0)
    k_late = _kkt_residual(small, oracle.solve(small, prm, x0, 10000, 0.0)[0], 1.0, 1.0)
    assert k_late < 1e-6 * k_early and k_late < 1e-7


# ---- T12 ----------------------------------------------------------------------

def test_zero_u_keeps_previous_p():
    g = synth.random_graph(6, 10, seed=31, isolated=1)  # vertex 5 has no edges
    st = _state(g, 32)
    i = g.n - 1
    st["p"][i] = [1.0, 0, 0, 0]
    st["q"][i] = [1.0, 0, 0, 0]
    prm = oracle.make_params(beta1=1.0, beta2=1.0, tau=1.5, gamma=(1.0, 1e-3, 1e-3, 1e-3))
    st["lam"][i] = [-2.0, 0, 0, 0]  # u_i = beta1 q_i + lam_i + gamma1 p_i = 0 exactly
    new, _, nz = oracle.iterate(g, prm, st)
    assert nz == 1
    np.testing.assert_array_equal(new["p"][i], st["p"][i])


# ---- odometry initialisation ----------------------------------------------------

def test_odometry_init_recovers_noise_free_truth():
    g = synth.random_walk_graph(80, n_closures=50, sigma_r=0.0, sigma_t=0.0, seed=41)
    q, t = oracle.init_odometry(g)
    # pose 0 of the walk is the identity at the origin
    sign = np.sign(np.sum(q * g.q_gt, axis=1, keepdims=True))
    assert np.abs(sign * q - g.q_gt).max() < 1e-12
    assert np.abs(t - g.t_gt).max() < 1e-11


def test_odometry_init_forest_roots():
    # two components; edges given in reverse direction exercise the q_e^* branch
    g = synth.random_graph(10, 0, seed=42)
    src = np.array([1, 2, 4, 7, 8], dtype=np.int32)
    dst = np.array([0, 1, 3, 6, 7], dtype=np.int32)
    q_gt = synth.random_unit_quaternions(np.random.default_rng(3), 10)
    t_gt = np.random.default_rng(4).standard_normal((10, 3))
    qm, tm = synth.measure(np.random.default_rng(5), q_gt, t_gt, src, dst, 0.0, 0.0)
    g = synth.PoseGraph(n=10, src=src, dst=dst, q_meas=qm, t_meas=tm, kappa=np.ones(5), omega=np.ones(5))
    q, t = oracle.init_odometry(g)
    # roots (lowest vertex per component) get the identity pose; isolated vertices too
    for r in (0, 3, 5, 6, 9):
        np.testing.assert_array_equal(q[r], [1, 0, 0, 0])
        np.testing.assert_array_equal(t[r], [0, 0, 0])
    # relative poses along the forest reproduce the noise-free measurements
    for e in range(5):
        i, j = src[e], dst[e]
        rel = synth._qmul(synth._qconj(q[i]), q[j])
        assert min(np.abs(rel - qm[e]).max(), np.abs(rel + qm[e]).max()) < 1e-12
        np.testing.assert_allclose(synth._rotate(synth._qconj(q[i]), t[j] - t[i]), tm[e], atol=1e-12)


# ---- inertial variant (reading R27: anchors x^k + theta (x^k - x^{k-1})) ------

THETA = 0.45


def _prev(g, seed):
    pv = synth.random_state(np.random.default_rng(seed), g.n)
    return {k: pv[k] for k in ("p", "q", "t", "s")}


def test_inertial_with_zero_theta_is_plain():
    g = synth.random_graph(20, 70, seed=3, isolated=1)
    st = _state(g, 3)
    a, res_a, _ = oracle.iterate(g, P(), st, 4)
    b, _, res_b, _ = oracle.iterate_inertial(g, P(), st, 0.0, 4, _prev(g, 4))
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])
    np.testing.assert_array_equal(res_a, res_b)


@pytest.mark.parametrize("gi", [0, 1, 2])
def test_inertial_blocks_minimise_with_extrapolated_anchors(gi):
    # every block of one inertial iteration minimises its subproblem of L_beta
    # plus 1/2 gamma |x - a|^2 around the extrapolated anchor a, formed here
    # from x^k and x^{k-1}; the returned previous iterate is x^k
    g = list(_graphs())[gi]
    st = _state(g, 40 + gi)
    pv = _prev(g, 50 + gi)
    new, pv_out, _, _ = oracle.iterate_inertial(g, P(), st, THETA, 1, pv)
    for k in ("p", "q", "t", "s"):
        np.testing.assert_array_equal(pv_out[k], st[k])
    anchor = {k: st[k] + THETA * (st[k] - pv[k]) for k in ("p", "q", "t", "s")}
    x_p, x_q, x_t, x_s = _blocks(g, st, new)
    rng = np.random.default_rng(9)
    cloud = rng.standard_normal((2000, 4))
    cloud /= np.linalg.norm(cloud, axis=1, keepdims=True)
    for i in range(g.n):
        f = lambda v: _obj(g, x_p, "p", i, v, anchor["p"][i], GAMMA[0])
        p_star = new["p"][i]
        f_star = f(p_star)
        assert f_star <= min(f(v) for v in cloud) + 1e-12
        h = 1e-5
        grad = np.array([(f(p_star + h * e) - f(p_star - h * e)) / (2 * h) for e in np.eye(4)])
        rg = grad - p_star * (p_star @ grad)
        assert np.linalg.norm(rg) < 1e-6 * max(1.0, np.linalg.norm(grad))
    for key, base, gam, dim in (("q", x_q, GAMMA[1], 4), ("t", x_t, GAMMA[2], 3), ("s", x_s, GAMMA[3], 3)):
        for i in range(g.n):
            v = new[key][i]
            f = lambda w: _obj(g, base, key, i, w, anchor[key][i], gam)
            h = 1e-3
            grad = np.array([(f(v + h * e) - f(v - h * e)) / (2 * h) for e in np.eye(dim)])
            assert np.linalg.norm(grad) < 1e-7 * max(1.0, abs(f(v))), (key, i, grad)


def test_inertial_noise_free_truth_is_fixed_point():
    for g in _noise_free_graphs():
        st = oracle.init_state(g.q_gt, g.t_gt)
        pv = {"p": g.q_gt, "q": g.q_gt, "t": g.t_gt, "s": g.t_gt}
        new, _, res, _ = oracle.iterate_inertial(g, P(), st, THETA, 3, pv)
        assert res[0] < 1e-24
        for k in ("p", "q"):
            np.testing.assert_allclose(new[k], g.q_gt, atol=1e-12)
        for k in ("t", "s"):
            np.testing.assert_allclose(new[k], g.t_gt, atol=1e-12)
