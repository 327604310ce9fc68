"""Second statement of one PRADMM iteration -- TEST INFRASTRUCTURE.

Built from the literal 4x4 matrices of Appendix A.2 (M(.), W(.),
D = diag(1,-1,-1,-1)) and the A_{s,i}, b_{s,i} of Appendix B, assembled per
vertex as printed (with readings R1 -- the in-edge matrix of the p-block is
W(q_li) W(q_l) D -- and R3 -- c_e uses the tail of e).  The C oracle uses the
equivalent quaternion-product forms instead; the two must agree to rounding.

Pure numpy, loops over vertices and edges, small graphs only.
"""
from __future__ import annotations

import numpy as np

D = np.diag([1.0, -1.0, -1.0, -1.0])
ONE = np.array([1.0, 0.0, 0.0, 0.0])


def M(a):
    """Left-multiplication matrix: M(a) b = a b (Appendix A.2)."""
    a0, a1, a2, a3 = a
    return np.array([[a0, -a1, -a2, -a3],
                     [a1, a0, -a3, a2],
                     [a2, a3, a0, -a1],
                     [a3, -a2, a1, a0]], dtype=np.float64)


def W(a):
    """Right-multiplication matrix: W(b) a = a b (Appendix A.2)."""
    a0, a1, a2, a3 = a
    return np.array([[a0, -a1, -a2, -a3],
                     [a1, a0, a3, -a2],
                     [a2, -a3, a0, a1],
                     [a3, a2, -a1, a0]], dtype=np.float64)


def pure(t3):
    return np.array([0.0, t3[0], t3[1], t3[2]])


def iterate(g, beta1, beta2, tau, gamma, st, check_scalar=True):
    """One iteration of Eq. (3a)-(3f) with the matrices of Appendix B.
    Returns (new_state, e^{k+1}, dict of the assembled A matrices' max
    off-scalar deviation)."""
    n, m = g.n, g.src.shape[0]
    src, dst = g.src.astype(np.int64), g.dst.astype(np.int64)
    qe, te, ka, om = g.q_meas, g.t_meas, g.kappa, g.omega
    p, q, t, s = st["p"].copy(), st["q"].copy(), st["t"].copy(), st["s"].copy()
    lam, z = st["lam"].copy(), st["z"].copy()
    g1, g2, g3, g4 = gamma
    out_of = [[] for _ in range(n)]
    in_of = [[] for _ in range(n)]
    for e in range(m):
        out_of[src[e]].append(e)
        in_of[dst[e]].append(e)
    dev = {"A1": 0.0, "A2": 0.0}

    # (3a) p-block, Appendix B.1
    p_new = p.copy()
    for i in range(n):
        A1 = (beta1 + g1) * np.eye(4)
        b1 = -beta1 * q[i] - lam[i] - g1 * p[i]
        for e in out_of[i]:
            j = dst[e]
            G1 = M(q[i]) @ M(pure(te[e])) @ D
            r = pure(t[j]) - pure(s[i])
            A1 += 2.0 * om[e] * G1.T @ G1
            b1 += -2.0 * om[e] * G1.T @ r
        for e in in_of[i]:
            l = src[e]
            G2 = W(qe[e]) @ W(q[l]) @ D
            A1 += 2.0 * ka[e] * G2.T @ G2
            b1 += -2.0 * ka[e] * G2.T @ ONE
        dev["A1"] = max(dev["A1"], np.abs(A1 - A1[0, 0] * np.eye(4)).max())
        nb = np.linalg.norm(b1)
        if nb > 0:
            p_new[i] = -b1 / nb
    p = p_new

    # (3b) q-block, Appendix B.2
    q_new = q.copy()
    for i in range(n):
        A2 = (beta1 + g2) * np.eye(4)
        b2 = beta1 * p[i] - lam[i] + g2 * q[i]
        for e in out_of[i]:
            j = dst[e]
            G3 = W(p[i]).T @ W(pure(te[e]))
            G4 = W(qe[e]) @ M(p[j]).T
            r = pure(t[j]) - pure(s[i])
            A2 += 2.0 * (om[e] * G3.T @ G3 + ka[e] * G4.T @ G4)
            b2 += 2.0 * (om[e] * G3.T @ r + ka[e] * G4.T @ ONE)
        dev["A2"] = max(dev["A2"], np.abs(A2 - A2[0, 0] * np.eye(4)).max())
        q_new[i] = np.linalg.solve(A2, b2)
    q_old = q
    q = q_new

    # c_e = Im(q_i t~_e p_i^*) = Im(M(q_i) M(t~_e) D p_i) for e = (i, j)
    c = np.zeros((m, 3))
    for e in range(m):
        i = src[e]
        c[e] = (M(q[i]) @ M(pure(te[e])) @ D @ p[i])[1:]

    # (3c) t-block, Appendix B.3
    t_new = t.copy()
    for i in range(n):
        A3 = (beta2 + g3) * np.eye(3)
        b3 = beta2 * s[i] + z[i] + g3 * t[i]
        for e in in_of[i]:
            l = src[e]
            A3 += 2.0 * om[e] * np.eye(3)
            b3 += 2.0 * om[e] * (s[l] + c[e])
        t_new[i] = np.linalg.solve(A3, b3)
    t_old = t
    t = t_new

    # (3d) s-block, Appendix B.4
    s_new = s.copy()
    for i in range(n):
        A4 = (beta2 + g4) * np.eye(3)
        b4 = beta2 * t[i] - z[i] + g4 * s[i]
        for e in out_of[i]:
            j = dst[e]
            A4 += 2.0 * om[e] * np.eye(3)
            b4 += 2.0 * om[e] * (t[j] - c[e])
        s_new[i] = np.linalg.solve(A4, b4)
    s = s_new

    # (3e), (3f)
    lam_new = lam - tau * beta1 * (p - q)
    z_new = z - tau * beta2 * (t - s)
    e_res = (np.sum((lam_new - lam) ** 2) / beta1 + np.sum((z_new - z) ** 2) / beta2
             + beta1 * np.sum((q - q_old) ** 2) + beta2 * np.sum((t - t_old) ** 2))
    new = {"p": p, "q": q, "t": t, "s": s, "lam": lam_new, "z": z_new}
    return new, float(e_res), dev
