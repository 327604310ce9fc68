"""Anchor-pose translation loss for the reverse mode, in torch.

Eq. (1) is invariant under a global rigid motion of all poses, so poses are
compared with ground truth in the frame of pose 0:

    L(p, t) = sum_i | R(p_0)^T (t_i - t_0) - R(q0_gt)^T (t_i_gt - t0_gt) |^2,

with R(p)^T v = Im(p^* [0, v] p) (Appendix A.2).  A loss head for
`pradmm.unrolled_poses`: torch differentiates it, and the library's reverse
sweeps take dL/dp, dL/dt from there.
"""
from __future__ import annotations


def _qmul(a, b):
    import torch
    w1, x1, y1, z1 = a.unbind(-1)
    w2, x2, y2, z2 = b.unbind(-1)
    return torch.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                        w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], -1)


def _rot_inv(q, v):
    """Im(q^* [0, v] q) for one quaternion q (4,) and vectors v (n, 3)."""
    import torch
    qc = q * torch.tensor([1.0, -1.0, -1.0, -1.0], dtype=q.dtype, device=q.device)
    vq = torch.cat([torch.zeros_like(v[:, :1]), v], -1)
    return _qmul(_qmul(qc.expand(v.shape[0], 4), vq), q.expand(v.shape[0], 4))[:, 1:]


def anchor_loss(p, t, q_gt, t_gt):
    """p (n x 4), t (n x 3) torch tensors; q_gt, t_gt ground truth (same device)."""
    d = _rot_inv(q_gt[0], t_gt - t_gt[0])
    y = _rot_inv(p[0], t - t[0]) - d
    return (y * y).sum()
