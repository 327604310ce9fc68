"""Vertex-partitioned plain PRADMM across ranks: the partition, the halo plan
and the exchanges of one iteration (host logic, one process per rank).

Every block of Algorithm 1 (Section 3.2, Eq. (3a)-(3f)) is Jacobi over
vertices, so a rank that owns a contiguous range of vertices can update them
if it holds, besides its own rows, the rows of the neighbours its vertices
read: its ghosts.  A rank keeps a local graph of its owned vertices followed
by its ghosts, with every edge that has an owned endpoint (in input order, so
each owned vertex sums its edges in the same order as the single-rank
iteration).  Ghost rows computed locally are partial and are never read
before an exchange refreshes them.

What each block reads from other vertices (Eq. (3) with the closed forms of
Appendix B):
  p-block  t_j over out-edges, q_l over in-edges          (x^k)
  q-block  t_j and p_j^{k+1} over out-edges
  c_e      q_l^{k+1}, p_l^{k+1} of the tail
  t-block  s_l^k and c_e over in-edges
  s-block  t_j^{k+1} over out-edges
so one iteration needs three exchanges:
  P_OUT   p^{k+1} of out-ghosts            after the p-block
  QPS_IN  q^{k+1}, p^{k+1}, s^k of in-ghosts after the q-block
  T_OUT   t^{k+1} of out-ghosts             after the t-block
(an out-ghost is the head of an owned vertex's out-edge, an in-ghost the
tail of an in-edge).  The p-block of the next iteration finds t^{k+1} of its
out-ghosts (T_OUT) and q^{k+1} of its in-ghosts (QPS_IN) already in place,
so the t and q exchanges before the p-block that a schedule of four
exchanges would make are folded into these.  The residual's four sums of
squares are all-reduced (32 bytes).

Every rank derives the whole plan from the edge list alone, so the plans of
all ranks agree without communication: what rank r sends to rank q of a
kind is the sorted list of q's ghosts of that kind that r owns, which is
exactly what q expects from r, in the same order.
"""
from __future__ import annotations

import numpy as np

P_OUT, QPS_IN, T_OUT = "P_OUT", "QPS_IN", "T_OUT"
KINDS = (P_OUT, QPS_IN, T_OUT)
# the state arrays each exchange carries, with their widths
CARRIES = {P_OUT: (("p", 4),), QPS_IN: (("q", 4), ("p", 4), ("s", 3)), T_OUT: (("t", 3),)}
WIDTH = {"p": 4, "q": 4, "t": 3, "s": 3, "lam": 4, "z": 3}


def partition(n: int, src, dst, world: int) -> list[tuple[int, int]]:
    """Contiguous vertex ranges [lo, hi), one per rank, balanced by work:
    a vertex weighs 1 plus its out- and in-degree.  Ranges in vertex order
    keep a walk's odometry neighbours together, so few edges are cut."""
    if world < 1:
        raise ValueError("world must be >= 1")
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    w = 1 + np.bincount(src, minlength=n) + np.bincount(dst, minlength=n)
    cum = np.concatenate([[0], np.cumsum(w)])
    cuts = [0]
    for r in range(1, world):
        cuts.append(int(np.searchsorted(cum, cum[-1] * r / world, side="left")))
    cuts.append(n)
    cuts = np.maximum.accumulate(np.minimum(np.array(cuts), n))
    return [(int(cuts[r]), int(cuts[r + 1])) for r in range(world)]


def _owner(ranges, v):
    los = np.array([lo for lo, _ in ranges])
    return np.searchsorted(los, v, side="right") - 1


class HaloPlan:
    """Rank `rank`'s local graph and exchange lists.

    Attributes:
      lo, hi        owned global vertex range
      verts         global ids of the local vertices: owned, then ghosts
      n_local       len(verts); the first hi - lo are owned
      edges         global ids of the local edges (an owned endpoint), input order
      src, dst      their endpoints as local ids (int32)
      send[kind]    {peer: local ids of owned rows that peer receives}
      recv[kind]    {peer: local ids of ghost rows filled from peer}
    """

    def __init__(self, n: int, src, dst, ranges, rank: int):
        src = np.asarray(src, dtype=np.int64)
        dst = np.asarray(dst, dtype=np.int64)
        self.ranges = [tuple(r) for r in ranges]
        self.rank = rank
        self.lo, self.hi = self.ranges[rank]
        ghosts = {}
        for r, (lo, hi) in enumerate(self.ranges):
            out_g = np.unique(dst[(src >= lo) & (src < hi) & ((dst < lo) | (dst >= hi))])
            in_g = np.unique(src[(dst >= lo) & (dst < hi) & ((src < lo) | (src >= hi))])
            ghosts[r] = {P_OUT: out_g, QPS_IN: in_g, T_OUT: out_g}
        own = (src >= self.lo) & (src < self.hi)
        own_h = (dst >= self.lo) & (dst < self.hi)
        self.edges = np.nonzero(own | own_h)[0]
        mine = ghosts[rank]
        ghost_ids = np.union1d(mine[P_OUT], mine[QPS_IN])
        self.verts = np.concatenate([np.arange(self.lo, self.hi), ghost_ids]).astype(np.int64)
        self.n_owned = self.hi - self.lo
        self.n_local = int(self.verts.size)
        g2l = np.full(n, -1, dtype=np.int64)
        g2l[self.verts] = np.arange(self.n_local)
        self._g2l = g2l
        self.src = g2l[src[self.edges]].astype(np.int32)
        self.dst = g2l[dst[self.edges]].astype(np.int32)
        self.send = {k: {} for k in KINDS}
        self.recv = {k: {} for k in KINDS}
        for kind in KINDS:
            ow = _owner(self.ranges, mine[kind]) if mine[kind].size else np.zeros(0, np.int64)
            for peer in range(len(self.ranges)):
                if peer == rank:
                    continue
                r_ids = mine[kind][ow == peer]
                if r_ids.size:
                    self.recv[kind][peer] = g2l[r_ids]
                theirs = ghosts[peer][kind]
                s_ids = theirs[(theirs >= self.lo) & (theirs < self.hi)]
                if s_ids.size:
                    self.send[kind][peer] = g2l[s_ids]

    def local_rows(self, global_arrays: dict) -> dict:
        """The local rows (owned, then ghosts) of full-size state arrays."""
        return {k: np.ascontiguousarray(np.asarray(v)[self.verts], dtype=np.float64) for k, v in global_arrays.items()}

    def halo_bytes(self) -> dict:
        """FP64 bytes this rank sends per iteration, by exchange."""
        out = {}
        for kind in KINDS:
            rows = sum(int(v.size) for v in self.send[kind].values())
            out[kind] = rows * sum(w for _, w in CARRIES[kind]) * 8
        return out


def exchange(plan: HaloPlan, kind: str, state: dict, group=None) -> None:
    """Refreshes the ghost rows of `kind` in the local state arrays (numpy,
    float64) from their owners: one send and one receive per peer, issued
    together, then waited on."""
    import torch
    import torch.distributed as dist

    arrays = CARRIES[kind]
    ops, inbox = [], {}
    for peer, ids in plan.send[kind].items():
        buf = np.concatenate([state[name][ids].reshape(-1) for name, _ in arrays])
        ops.append(dist.P2POp(dist.isend, torch.from_numpy(buf), peer, group))
    for peer, ids in plan.recv[kind].items():
        t = torch.empty(int(ids.size) * sum(w for _, w in arrays), dtype=torch.float64)
        inbox[peer] = t
        ops.append(dist.P2POp(dist.irecv, t, peer, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    for peer, t in inbox.items():
        ids = plan.recv[kind][peer]
        buf = t.numpy()
        off = 0
        for name, w in arrays:
            k = int(ids.size) * w
            state[name][ids] = buf[off:off + k].reshape(-1, w)
            off += k


def iterate_partitioned(plan: HaloPlan, block, state: dict, betas: tuple[float, float], group=None):
    """One iteration of plain PRADMM on this rank's local graph.

    block(which, state) runs one block of Algorithm 1 on the local graph in
    place: which = "p", "q", "c", "t", "s", "duals" (c carries c_e from "c"
    to "t" and "s").  state holds the local rows of p, q, t, s, lam, z with
    up-to-date ghosts of x^k.  Returns e^{k+1} (Appendix E.1 with beta1 for
    the lambda / q terms and beta2 for the z / t terms), summed over the
    owned rows of all ranks."""
    import torch
    import torch.distributed as dist

    k = plan.n_owned
    old = {name: state[name][:k].copy() for name in ("q", "t", "lam", "z")}
    block("p", state)
    exchange(plan, P_OUT, state, group)
    block("q", state)
    exchange(plan, QPS_IN, state, group)
    block("c", state)
    block("t", state)
    exchange(plan, T_OUT, state, group)
    block("s", state)
    block("duals", state)
    d = lambda name: float(np.sum((state[name][:k] - old[name]) ** 2))
    parts = torch.tensor([d("lam"), d("z"), d("q"), d("t")], dtype=torch.float64)
    dist.all_reduce(parts, group=group)
    dl, dz, dq, dt = (float(x) for x in parts)
    b1, b2 = betas
    return dl / b1 + dz / b2 + b1 * dq + b2 * dt
