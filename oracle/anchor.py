"""Anchor-pose translation loss and its gradient, FP64 numpy -- TEST
INFRASTRUCTURE (used with the oracle's reverse mode).

Eq. (1) is invariant under a global rigid motion of all poses, so poses are
compared with ground truth in the frame of pose 0:

    L(p, t) = sum_i | R(p_0)^T (t_i - t_0) - R(q0_gt)^T (t_i_gt - t0_gt) |^2,

with R(p)^T v = Im(p^* [0, v] p) (Appendix A.2), which is the inverse rotation
for a unit p.  `anchor_loss` returns L, dL/dp (only row 0 is non-zero) and
dL/dt, written from the product rule of the quaternion products.
"""
from __future__ import annotations

import numpy as np


def _qmul(a, b):
    w1, x1, y1, z1 = np.moveaxis(a, -1, 0)
    w2, x2, y2, z2 = np.moveaxis(b, -1, 0)
    return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], -1)


def _conj(a):
    return a * np.array([1.0, -1.0, -1.0, -1.0])


def _pure(v):
    return np.concatenate([np.zeros(v.shape[:-1] + (1,)), v], -1)


def anchor_loss(p, t, q_gt, t_gt):
    """Returns (L, dL/dp (n x 4), dL/dt (n x 3))."""
    p, t = np.asarray(p, dtype=np.float64), np.asarray(t, dtype=np.float64)
    q_gt, t_gt = np.asarray(q_gt, dtype=np.float64), np.asarray(t_gt, dtype=np.float64)
    d = _qmul(_qmul(_conj(q_gt[0]), _pure(t_gt - t_gt[0])), q_gt[0])[:, 1:]
    v = t - t[0]
    y = _qmul(_qmul(_conj(p[0]), _pure(v)), p[0])[:, 1:] - d
    L = float((y * y).sum())
    # y_i = Im(p0^* v~_i p0) - d_i:  dy/dv is v -> Im(p0^* v~ p0), whose
    # transpose is y -> Im(p0 y~ p0^*); dy/dp0 has transpose -2 v~_i p0 Ybar_i
    Yb = _pure(2.0 * y)
    gt = _qmul(_qmul(p[0], Yb), _conj(p[0]))[:, 1:]
    dt = gt.copy()
    dt[0] -= gt.sum(0)
    dp = np.zeros_like(p)
    dp[0] = (-2.0 * _qmul(_qmul(_pure(v), p[0]), Yb)).sum(0)
    return L, dp, dt
