"""PRADMM with general weight matrices Sigma_1, Sigma_2 -- TEST INFRASTRUCTURE.

Only the test suite may import this module.  It shares no code with the
CUDA library.

Model (1) / split model (2) with ||.||_{Sigma} norms: edge e = (i, j) weighs
the translation residual with omega_e Sigma_1 and the rotation residual with
kappa_e Sigma_2, where Sigma_1, Sigma_2 are symmetric positive definite 4x4
matrices shared by all edges (Section 2 writes one Sigma_1 and one Sigma_2;
the per-edge scalars are reading R9).  With Sigma_1 = Sigma_2 = I this is the
scalar model of the C oracle.

Every block follows Appendix B with the literal 4x4 matrices of Appendix A.2:
  p-block (3a): A_1 = 2 sum_out w G1^T S1 G1 + 2 sum_in k G2^T S2 G2 + (beta1 + gamma1) I,
                b_1 = -2 sum_out w G1^T S1 r~ - 2 sum_in k G2^T S2 1~ - beta1 q - lam - gamma1 p,
                G1 = M(q_i) M(t~_e) D, G2 = W(q_e) W(q_l) D (reading R1), r~ = t~_j - s~_i,
                p = argmin_{|p| = 1} 1/2 p^T A_1 p + b_1^T p          (Lemma 1, Algorithm 2)
  q-block (3b): q = A_2^{-1} b_2 with G3 = W(p_i^*) W(t~_e), G4 = M(p_j^*) W(q_e),
                A_2 = 2 sum_out (w G3^T S1 G3 + k G4^T S2 G4) + (beta1 + gamma2) I,
                b_2 = 2 sum_out (w G3^T S1 r~ + k G4^T S2 1~) + beta1 p - lam + gamma2 q
  t-block (3c): t = A_3^{-1} b_3, E = [0; I_3] embeds R^3 as pure quaternions,
                A_3 = 2 sum_in w E^T S1 E + (beta2 + gamma3) I,
                b_3 = 2 sum_in w E^T S1 (s~_l + c~_e) + beta2 s + z + gamma3 t,
                c~_e = q_l t~_e p_l^* (the whole quaternion: with a general S1 its real
                part couples to the translation through S1's off-diagonal entries)
  s-block (3d): s = A_4^{-1} b_4,  A_4 = 2 sum_out w E^T S1 E + (beta2 + gamma4) I,
                b_4 = 2 sum_out w E^T S1 (t~_j - c~_e) - z + beta2 t + gamma4 s
  duals (3e, 3f) and the residual of Appendix E.1 as in the scalar case.
The gamma terms above are the proximal terms around x^k; the inertial variant
(reading R27) puts them around x^{k+1/2} = x^k + theta (x^k - x^{k-1}), the
anchors Appendix B writes, for p, q, t and s.

The p-block's sphere-constrained quadratic is solved by Algorithm 2: lambda*
is the rightmost real eigenvalue of Q y = -lambda y with
Q = [[A, -b b^T], [-I, A]], and p = -(A + lambda* I)^{-1} b.  When A + lambda* I
is singular (the hard case of the Appendix C lemma: lambda* = -a_min and b
orthogonal to its eigenvectors) the solution is -(A + lambda* I)^+ b plus the
multiple of an eigenvector of a_min that restores |p| = 1; of the two signs
the one closer to p^k is kept (reading R24: both minimise, the paper does not
choose).

Pure numpy, per-vertex loops: small graphs only.
"""
from __future__ import annotations

import numpy as np

from .matrix_form import D, M, ONE, W, pure

E3 = np.vstack([np.zeros((1, 3)), np.eye(3)])  # R^3 -> pure quaternions


def conj(a):
    return D @ a


def trs_sphere(A, b, x_prev=None):
    """argmin_{|x| = 1} 1/2 x^T A x + b^T x (Lemma 1 / Algorithm 2).
    Returns (x, lambda*, hard) with (A + lambda* I) x = -b, A + lambda* I >= 0."""
    A = 0.5 * (A + A.T)
    n = A.shape[0]
    Q = np.block([[A, -np.outer(b, b)], [-np.eye(n), A]])
    mu = np.linalg.eigvals(Q)
    scale = max(1.0, np.abs(A).max(), float(b @ b))
    real = mu[np.abs(mu.imag) <= 1e-7 * scale].real
    lam = float(-real.min())
    a, V = np.linalg.eigh(A)
    lam = max(lam, -a[0])  # A + lambda I >= 0 (rounding can put lambda* a hair below)
    K = A + lam * np.eye(n)
    gap = a + lam  # eigenvalues of K
    if gap[0] > 1e-9 * scale:
        x = -np.linalg.solve(K, b)
        if abs(np.linalg.norm(x) - 1.0) <= 1e-6:
            return x, lam, False
    # hard case: lambda* = -a_min, b has no component on the a_min eigenspace
    # (there lambda* is a defective eigenvalue of Q, found only to ~sqrt(eps))
    lam = -float(a[0])
    gap = a - a[0]
    null = gap <= 1e-7 * scale
    g = V.T @ b
    xp = -(V[:, ~null] @ (g[~null] / gap[~null]))
    alpha = np.sqrt(max(0.0, 1.0 - float(xp @ xp)))
    v = V[:, null][:, 0]
    x1, x2 = xp + alpha * v, xp - alpha * v
    if x_prev is not None and np.linalg.norm(x2 - x_prev) < np.linalg.norm(x1 - x_prev):
        x1 = x2
    return x1, lam, True


def p_system(g, params, Sigma1, Sigma2, st, i):
    """A_1 and b_1 of the p-block of vertex i (Appendix B.1), as assembled in
    `iterate`."""
    beta1, _, _, gam = params
    S1, S2 = np.asarray(Sigma1, dtype=np.float64), np.asarray(Sigma2, dtype=np.float64)
    p, q, t, s, lam = st["p"], st["q"], st["t"], st["s"], st["lam"]
    A1 = (beta1 + gam[0]) * np.eye(4)
    b1 = -beta1 * q[i] - lam[i] - gam[0] * p[i]
    for e in np.nonzero(g.src == i)[0]:
        G1 = M(q[i]) @ M(pure(g.t_meas[e])) @ D
        r = pure(t[g.dst[e]]) - pure(s[i])
        A1 += 2.0 * g.omega[e] * G1.T @ S1 @ G1
        b1 -= 2.0 * g.omega[e] * G1.T @ S1 @ r
    for e in np.nonzero(g.dst == i)[0]:
        G2 = W(g.q_meas[e]) @ W(q[g.src[e]]) @ D
        A1 += 2.0 * g.kappa[e] * G2.T @ S2 @ G2
        b1 -= 2.0 * g.kappa[e] * G2.T @ S2 @ ONE
    return A1, b1


def iterate(g, params, Sigma1, Sigma2, st, anchors=None):
    """One iteration of Eq. (3a)-(3f) with weights omega_e Sigma1, kappa_e Sigma2.
    params: (beta1, beta2, tau, (gamma1..gamma4)).  `anchors` (p, q, t, s) are
    the proximal anchors x^{k+1/2} of Appendix B; None means x^k (plain
    PRADMM).  Returns (new_state, e^{k+1}, number of hard-case p-updates)."""
    beta1, beta2, tau, gam = params
    g1, g2, g3, g4 = gam
    S1, S2 = np.asarray(Sigma1, dtype=np.float64), np.asarray(Sigma2, dtype=np.float64)
    n, m = g.n, g.src.shape[0]
    src, dst = g.src.astype(np.int64), g.dst.astype(np.int64)
    qe, te, ka, om = g.q_meas, g.t_meas, g.kappa, g.omega
    p, q, t, s = (st[k].copy() for k in ("p", "q", "t", "s"))
    lam, z = st["lam"].copy(), st["z"].copy()
    if anchors is None:
        ap, aq, at, as_ = p, q, t, s
    else:
        ap, aq, at, as_ = (np.asarray(anchors[k], dtype=np.float64) for k in ("p", "q", "t", "s"))
    out_of = [[] for _ in range(n)]
    in_of = [[] for _ in range(n)]
    for e in range(m):
        out_of[src[e]].append(e)
        in_of[dst[e]].append(e)
    hard = 0

    # (3a) p-block
    pn = p.copy()
    for i in range(n):
        A1 = (beta1 + g1) * np.eye(4)
        b1 = -beta1 * q[i] - lam[i] - g1 * ap[i]
        for e in out_of[i]:
            G1 = M(q[i]) @ M(pure(te[e])) @ D
            r = pure(t[dst[e]]) - pure(s[i])
            A1 += 2.0 * om[e] * G1.T @ S1 @ G1
            b1 -= 2.0 * om[e] * G1.T @ S1 @ r
        for e in in_of[i]:
            G2 = W(qe[e]) @ W(q[src[e]]) @ D
            A1 += 2.0 * ka[e] * G2.T @ S2 @ G2
            b1 -= 2.0 * ka[e] * G2.T @ S2 @ ONE
        pn[i], _, h = trs_sphere(A1, b1, p[i])
        hard += int(h)
    p = pn

    # (3b) q-block
    qn = q.copy()
    for i in range(n):
        A2 = (beta1 + g2) * np.eye(4)
        b2 = beta1 * p[i] - lam[i] + g2 * aq[i]
        for e in out_of[i]:
            j = dst[e]
            G3 = W(conj(p[i])) @ W(pure(te[e]))
            G4 = M(conj(p[j])) @ W(qe[e])
            r = pure(t[j]) - pure(s[i])
            A2 += 2.0 * (om[e] * G3.T @ S1 @ G3 + ka[e] * G4.T @ S2 @ G4)
            b2 += 2.0 * (om[e] * G3.T @ S1 @ r + ka[e] * G4.T @ S2 @ ONE)
        qn[i] = np.linalg.solve(A2, b2)
    q_old, q = q, qn

    def c_full(e):
        i = src[e]
        return M(q[i]) @ M(pure(te[e])) @ conj(p[i])

    # (3c) t-block
    tn = t.copy()
    for i in range(n):
        A3 = (beta2 + g3) * np.eye(3)
        b3 = beta2 * s[i] + z[i] + g3 * at[i]
        for e in in_of[i]:
            w = pure(s[src[e]]) + c_full(e)
            A3 += 2.0 * om[e] * E3.T @ S1 @ E3
            b3 += 2.0 * om[e] * E3.T @ S1 @ w
        tn[i] = np.linalg.solve(A3, b3)
    t_old, t = t, tn

    # (3d) s-block
    sn = s.copy()
    for i in range(n):
        A4 = (beta2 + g4) * np.eye(3)
        b4 = beta2 * t[i] - z[i] + g4 * as_[i]
        for e in out_of[i]:
            w = pure(t[dst[e]]) - c_full(e)
            A4 += 2.0 * om[e] * E3.T @ S1 @ E3
            b4 += 2.0 * om[e] * E3.T @ S1 @ w
        sn[i] = np.linalg.solve(A4, b4)
    s = sn

    # (3e), (3f) and the residual of Appendix E.1
    lam_old, z_old = lam, z
    lam = lam - tau * beta1 * (p - q)
    z = z - tau * beta2 * (t - s)
    e_res = (np.sum((lam - lam_old) ** 2) / beta1 + np.sum((z - z_old) ** 2) / beta2
             + beta1 * np.sum((q - q_old) ** 2) + beta2 * np.sum((t - t_old) ** 2))
    return {"p": p, "q": q, "t": t, "s": s, "lam": lam, "z": z}, float(e_res), hard


def iterate_inertial(g, params, Sigma1, Sigma2, st, theta, prev=None):
    """One inertial iteration (reading R27): the anchors of Appendix B are
    x^{k+1/2} = x^k + theta (x^k - x^{k-1}) for x = p, q, t, s; `prev` holds
    x^{k-1} (None: x^{-1} = x^0).  The hard case's sign still follows p^k.
    Returns (new_state, new_prev = x^k, e^{k+1}, hard-case count)."""
    cur = {k: np.asarray(st[k], dtype=np.float64) for k in ("p", "q", "t", "s")}
    old = cur if prev is None else {k: np.asarray(prev[k], dtype=np.float64) for k in ("p", "q", "t", "s")}
    anchors = {k: cur[k] + theta * (cur[k] - old[k]) for k in cur}
    new, e_res, hard = iterate(g, params, Sigma1, Sigma2, st, anchors)
    return new, {k: cur[k].copy() for k in cur}, e_res, hard


def lagrangian(g, params, Sigma1, Sigma2, st):
    """Augmented Lagrangian of Section 3.2 with the Sigma-weighted split model (2)."""
    beta1, beta2, _, _ = params
    S1, S2 = np.asarray(Sigma1, dtype=np.float64), np.asarray(Sigma2, dtype=np.float64)
    p, q, t, s, lam, z = (st[k] for k in ("p", "q", "t", "s", "lam", "z"))
    L = 0.0
    for e in range(g.src.shape[0]):
        i, j = int(g.src[e]), int(g.dst[e])
        rho = pure(t[j]) - pure(s[i]) - M(q[i]) @ M(pure(g.t_meas[e])) @ conj(p[i])
        eta = M(conj(p[j])) @ M(q[i]) @ g.q_meas[e] - ONE
        L += g.omega[e] * rho @ S1 @ rho + g.kappa[e] * eta @ S2 @ eta
    L += -np.sum(lam * (p - q)) + 0.5 * beta1 * np.sum((p - q) ** 2)
    L += -np.sum(z * (t - s)) + 0.5 * beta2 * np.sum((t - s) ** 2)
    return float(L)


def objective(g, Sigma1, Sigma2, q, t):
    """F of Eq. (1) with the Sigma-weighted norms, at (q, t)."""
    S1, S2 = np.asarray(Sigma1, dtype=np.float64), np.asarray(Sigma2, dtype=np.float64)
    F = 0.0
    for e in range(g.src.shape[0]):
        i, j = int(g.src[e]), int(g.dst[e])
        rho = pure(t[j]) - pure(t[i]) - M(q[i]) @ M(pure(g.t_meas[e])) @ conj(q[i])
        eta = M(conj(q[j])) @ M(q[i]) @ g.q_meas[e] - ONE
        F += g.omega[e] * rho @ S1 @ rho + g.kappa[e] * eta @ S2 @ eta
    return float(F)
