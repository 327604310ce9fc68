"""Seeded synthetic pose graphs.

Inputs for the solver, its tests and its benchmark.  This module holds the
data model only -- ground-truth trajectories and the noisy relative
measurements of the generative model of Section 2 -- and none of the
iteration's arithmetic, so it can feed both the CUDA library and the FP64
oracle with byte-identical arrays.

Generative model (Section 2):
    t_ij = R_i^T (t_j - t_i) + t_eps,        t_eps ~ N(0, sigma_t^2 I_3)
    q_ij = q_i^* q_j q_eps
The paper draws q_eps from a von Mises-Fisher law whose printed concentration
(Section 5) is garbled; here q_eps is an axis-angle perturbation with its axis
uniform on S^2 and its angle ~ N(0, sigma_r), i.e. q_eps = [cos(a/2), sin(a/2) n].

Quaternions are scalar first.  Every array is C-contiguous: src, dst int32;
q_meas (m, 4), t_meas (m, 3), kappa (m,), omega (m,) float64; ground truth
q_gt (n, 4), t_gt (n, 3) float64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class PoseGraph:
    n: int
    src: np.ndarray
    dst: np.ndarray
    q_meas: np.ndarray
    t_meas: np.ndarray
    kappa: np.ndarray
    omega: np.ndarray
    q_gt: np.ndarray | None = None
    t_gt: np.ndarray | None = None
    name: str = ""
    info: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.src.shape[0])


# ---- quaternion helpers for the data model (vectorised, float64) -----------

def _qmul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    a0, a1, a2, a3 = a[..., 0], a[..., 1], a[..., 2], a[..., 3]
    b0, b1, b2, b3 = b[..., 0], b[..., 1], b[..., 2], b[..., 3]
    return np.stack([
        a0 * b0 - a1 * b1 - a2 * b2 - a3 * b3,
        a0 * b1 + a1 * b0 + a2 * b3 - a3 * b2,
        a0 * b2 - a1 * b3 + a2 * b0 + a3 * b1,
        a0 * b3 + a1 * b2 - a2 * b1 + a3 * b0,
    ], axis=-1)


def _qconj(a: np.ndarray) -> np.ndarray:
    return a * np.array([1.0, -1.0, -1.0, -1.0])


def _rotate(q: np.ndarray, v: np.ndarray) -> np.ndarray:
    vq = np.concatenate([np.zeros(v.shape[:-1] + (1,)), v], axis=-1)
    return _qmul(_qmul(q, vq), _qconj(q))[..., 1:]


def random_unit_quaternions(rng: np.random.Generator, k: int) -> np.ndarray:
    x = rng.standard_normal((k, 4))
    return x / np.linalg.norm(x, axis=1, keepdims=True)


def axis_angle_noise(rng: np.random.Generator, k: int, sigma_r: float) -> np.ndarray:
    """q_eps with axis uniform on S^2 and angle ~ N(0, sigma_r)."""
    axis = rng.standard_normal((k, 3))
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    ang = rng.standard_normal(k) * sigma_r
    return np.concatenate([np.cos(ang / 2)[:, None], np.sin(ang / 2)[:, None] * axis], axis=1)


def measure(rng: np.random.Generator, q_gt: np.ndarray, t_gt: np.ndarray, src: np.ndarray,
            dst: np.ndarray, sigma_r: float, sigma_t: float) -> tuple[np.ndarray, np.ndarray]:
    """Noisy relative measurements of the generative model of Section 2."""
    m = src.shape[0]
    qi, qj = q_gt[src], q_gt[dst]
    q_eps = axis_angle_noise(rng, m, sigma_r)
    q_meas = _qmul(_qmul(_qconj(qi), qj), q_eps)
    q_meas /= np.linalg.norm(q_meas, axis=1, keepdims=True)
    t_meas = _rotate(_qconj(qi), t_gt[dst] - t_gt[src]) + sigma_t * rng.standard_normal((m, 3))
    return np.ascontiguousarray(q_meas), np.ascontiguousarray(t_meas)


def _finish(name, n, src, dst, q_gt, t_gt, rng, sigma_r, sigma_t, info=None, weights=None):
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    q_meas, t_meas = measure(rng, q_gt, t_gt, src, dst, sigma_r, sigma_t)
    m = src.shape[0]
    if weights is None:
        kappa = np.ones(m)
        omega = np.ones(m)
    else:
        kappa, omega = weights
    return PoseGraph(n=n, src=src, dst=dst, q_meas=q_meas, t_meas=t_meas,
                     kappa=np.ascontiguousarray(kappa, dtype=np.float64),
                     omega=np.ascontiguousarray(omega, dtype=np.float64),
                     q_gt=np.ascontiguousarray(q_gt), t_gt=np.ascontiguousarray(t_gt),
                     name=name, info=dict(info or {}))


# ---- trajectories -----------------------------------------------------------

def yaw_pitch_walk(rng: np.random.Generator, n: int, turn: float = math.pi / 4):
    """Unit-step walk whose heading turns by yaw, pitch ~ U(-turn, turn) per step.

    The orientation of pose k is R_k = Rz(Y_k) Ry(P_k) with Y_k, P_k the sums
    of the turns so far; pose k+1 lies one metre along the heading R_{k+1} e_x.
    """
    yaw = np.concatenate([[0.0], rng.uniform(-turn, turn, n - 1)])
    pitch = np.concatenate([[0.0], rng.uniform(-turn, turn, n - 1)])
    Y = np.cumsum(yaw)
    P = np.cumsum(pitch)
    qz = np.stack([np.cos(Y / 2), np.zeros(n), np.zeros(n), np.sin(Y / 2)], axis=1)
    qy = np.stack([np.cos(P / 2), np.zeros(n), np.sin(P / 2), np.zeros(n)], axis=1)
    q = _qmul(qz, qy)
    heading = np.stack([np.cos(Y) * np.cos(P), np.sin(Y) * np.cos(P), -np.sin(P)], axis=1)
    heading[0] = 0.0
    t = np.cumsum(heading, axis=0)
    return q, t


def _pairs_within(t: np.ndarray, radius: float) -> np.ndarray:
    """All pairs (i, j), i < j - 1, with |t_i - t_j| < radius, sorted."""
    from scipy.spatial import cKDTree

    pairs = cKDTree(t).query_pairs(radius, output_type="ndarray")
    if pairs.size == 0:
        return np.zeros((0, 2), dtype=np.int64)
    pairs = np.sort(pairs.astype(np.int64), axis=1)
    pairs = pairs[pairs[:, 1] > pairs[:, 0] + 1]
    d = np.linalg.norm(t[pairs[:, 0]] - t[pairs[:, 1]], axis=1)
    pairs = pairs[d < radius]
    order = np.lexsort((pairs[:, 1], pairs[:, 0]))
    return pairs[order]


def random_walk_graph(n: int = 128, n_closures: int | None = 200, closure_density: float | None = None,
                      radius: float = 3.0, sigma_r: float = 0.05, sigma_t: float = 0.1,
                      seed: int = 1, name: str = "walk") -> PoseGraph:
    """Odometry chain of a yaw/pitch walk plus loop closures drawn uniformly,
    without replacement, among pose pairs closer than `radius`."""
    rng = np.random.default_rng(seed)
    q_gt, t_gt = yaw_pitch_walk(rng, n)
    cand = _pairs_within(t_gt, radius)
    want = n_closures if n_closures is not None else int(round(closure_density * n))
    k = min(want, cand.shape[0])
    pick = np.sort(rng.choice(cand.shape[0], size=k, replace=False)) if k > 0 else np.zeros(0, np.int64)
    cl = cand[pick]
    src = np.concatenate([np.arange(n - 1), cl[:, 0]])
    dst = np.concatenate([np.arange(1, n), cl[:, 1]])
    info = {"closures_requested": int(want), "closures": int(k), "candidates": int(cand.shape[0])}
    return _finish(name, n, src, dst, q_gt, t_gt, rng, sigma_r, sigma_t, info)


def helix_graph(n: int = 25000, radius: float = 10.0, pitch: float = 0.5, per_turn: int = 100,
                sigma_r: float = 0.01, sigma_t: float = 0.05, seed: int = 2) -> PoseGraph:
    """Helical trajectory, orientation tangent aligned; odometry edges plus a
    directed closure from every pose to the poses one turn above and below."""
    rng = np.random.default_rng(seed)
    k = np.arange(n, dtype=np.float64)
    phi = 2.0 * math.pi * k / per_turn
    t_gt = np.stack([radius * np.cos(phi), radius * np.sin(phi), pitch * k / per_turn], axis=1)
    climb = math.atan2(pitch, 2.0 * math.pi * radius)
    Y = phi + math.pi / 2
    qz = np.stack([np.cos(Y / 2), np.zeros(n), np.zeros(n), np.sin(Y / 2)], axis=1)
    qy = np.tile([math.cos(-climb / 2), 0.0, math.sin(-climb / 2), 0.0], (n, 1))
    q_gt = _qmul(qz, qy)
    idx = np.arange(n)
    up = idx[idx + per_turn < n]
    down = idx[idx >= per_turn]
    src = np.concatenate([idx[:-1], up, down])
    dst = np.concatenate([idx[1:], up + per_turn, down - per_turn])
    return _finish("helix", n, src, dst, q_gt, t_gt, rng, sigma_r, sigma_t)


def ring_graph(n: int = 100, radius: float = 2.0, sigma_r: float = 0.01, sigma_t: float = 0.01,
               seed: int = 7) -> PoseGraph:
    """The circular ring of the paper's synthetic experiments (Section 5): n
    poses on one planar loop of the given radius, orientation tangent to the
    loop, odometry edges (i, i+1) and the closing edge (n-1, 0), so m = n."""
    rng = np.random.default_rng(seed)
    phi = 2.0 * math.pi * np.arange(n, dtype=np.float64) / n
    t_gt = np.stack([radius * np.cos(phi), radius * np.sin(phi), np.zeros(n)], axis=1)
    Y = phi + math.pi / 2
    q_gt = np.stack([np.cos(Y / 2), np.zeros(n), np.zeros(n), np.sin(Y / 2)], axis=1)
    src = np.arange(n)
    dst = (src + 1) % n
    return _finish(f"ring{n}", n, src, dst, q_gt, t_gt, rng, sigma_r, sigma_t,
                   info={"radius": radius, "sigma_r": sigma_r, "sigma_t": sigma_t})


def cube_graph(side: int = 7, p_cube: float = 0.3, extent: float = 2.0, sigma_r: float = 0.1,
               sigma_t: float = 0.1, seed: int = 11) -> PoseGraph:
    """The cube dataset of the paper's synthetic experiments (Section 5): a
    robot visits every node of a side^3 grid spanning an extent^3 world along
    a serpentine path (odometry, side^3 - 1 edges); every pair of grid
    neighbours the path does not join gets each of its two directed closures
    independently with probability p_cube, which gives the paper's expected
    edge count E(m) = 2 (2 side^3 - 3 side^2 + 1) p_cube + side^3 - 1.
    Ground-truth orientations are uniform on SO(3)."""
    rng = np.random.default_rng(seed)
    # serpentine order: x varies fastest, reversing on alternate rows; rows
    # reverse on alternate layers, so consecutive nodes are grid neighbours
    order = []
    for z in range(side):
        ys = range(side) if z % 2 == 0 else range(side - 1, -1, -1)
        for row, y in enumerate(ys):
            xs = range(side) if (row + z * side) % 2 == 0 else range(side - 1, -1, -1)
            for x in xs:
                order.append((x, y, z))
    coords = np.array(order, dtype=np.float64)
    n = side ** 3
    step = extent / max(side - 1, 1)
    t_gt = coords * step
    q_gt = random_unit_quaternions(rng, n)
    pos = {c: k for k, c in enumerate(order)}
    path = {(k, k + 1) for k in range(n - 1)}
    src, dst = list(range(n - 1)), list(range(1, n))
    for (x, y, z), a in pos.items():
        for dx, dy, dz in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
            b = pos.get((x + dx, y + dy, z + dz))
            if b is None or (min(a, b), max(a, b)) in path:
                continue
            for u, v in ((a, b), (b, a)):
                if rng.random() < p_cube:
                    src.append(u)
                    dst.append(v)
    return _finish(f"cube{side}", n, np.array(src), np.array(dst), q_gt, t_gt, rng, sigma_r, sigma_t,
                   info={"side": side, "p_cube": p_cube, "extent": extent})


# axis-aligned headings of a lattice walk: +x, -x, +y, -y, +z, -z
_LATTICE_STEP = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])
_H = math.sqrt(0.5)
_LATTICE_Q = np.array([[1, 0, 0, 0], [0, 0, 0, 1], [_H, 0, 0, _H], [_H, 0, 0, -_H],
                       [_H, 0, -_H, 0], [_H, 0, _H, 0]], dtype=np.float64)


def lattice_walk_graph(n: int = 1_000_000, side: int = 100, p_closure: float = 0.3,
                       sigma_r: float = 0.02, sigma_t: float = 0.1, seed: int = 3) -> PoseGraph:
    """Random walk on a side^3 lattice (unit moves to a uniformly chosen
    in-bounds neighbour site), heading along the last move.  Closures: for each
    pose and each of its lattice-neighbour sites, every earlier pose at that
    site becomes an edge (earlier -> later) with probability p_closure; the pair
    already joined by odometry is skipped."""
    rng = np.random.default_rng(seed)
    pos = np.empty((n, 3), dtype=np.int64)
    mv = np.zeros(n, dtype=np.int64)
    x = [side // 2, side // 2, side // 2]
    pos[0] = x
    draws = rng.integers(0, 6, size=4 * n + 64)
    d_i = 0
    steps = _LATTICE_STEP.tolist()
    for k in range(1, n):
        while True:
            d = int(draws[d_i]); d_i += 1
            if d_i >= draws.shape[0]:
                draws = rng.integers(0, 6, size=n); d_i = 0
            s = steps[d]
            nx, ny, nz = x[0] + s[0], x[1] + s[1], x[2] + s[2]
            if 0 <= nx < side and 0 <= ny < side and 0 <= nz < side:
                break
        x = [nx, ny, nz]
        pos[k] = x
        mv[k] = d
    q_gt = _LATTICE_Q[mv].copy()
    q_gt[0] = [1.0, 0.0, 0.0, 0.0]
    t_gt = pos.astype(np.float64)

    site = pos[:, 0] + side * pos[:, 1] + side * side * pos[:, 2]
    order = np.argsort(site, kind="stable")  # poses grouped by site, by index inside a site
    site_sorted = site[order]
    start = np.searchsorted(site_sorted, np.arange(side ** 3), side="left")
    src_l, dst_l = [], []
    idx = np.arange(n)
    for s in _LATTICE_STEP:
        nb = pos + s
        ok = np.all((nb >= 0) & (nb < side), axis=1)
        i_ok = idx[ok]
        nb_site = nb[ok, 0] + side * nb[ok, 1] + side * side * nb[ok, 2]
        lo = start[nb_site]
        # earlier poses at the neighbour site: those with index < i
        hi = np.searchsorted(site_sorted * (n + 1) + order, nb_site * (n + 1) + i_ok, side="left")
        cnt = hi - lo
        tot = int(cnt.sum())
        if tot == 0:
            continue
        rep_i = np.repeat(i_ok, cnt)
        offs = np.arange(tot) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        j = order[np.repeat(lo, cnt) + offs]
        keep = rng.random(tot) < p_closure
        keep &= j != rep_i - 1
        src_l.append(j[keep])
        dst_l.append(rep_i[keep])
    cs = np.concatenate(src_l) if src_l else np.zeros(0, np.int64)
    cd = np.concatenate(dst_l) if dst_l else np.zeros(0, np.int64)
    o = np.lexsort((cd, cs))
    src = np.concatenate([np.arange(n - 1), cs[o]])
    dst = np.concatenate([np.arange(1, n), cd[o]])
    info = {"side": side, "p_closure": p_closure, "closures": int(cs.shape[0])}
    return _finish("lattice", n, src, dst, q_gt, t_gt, rng, sigma_r, sigma_t, info)


def random_graph(n: int, m: int, seed: int, weights: bool = True, isolated: int = 0,
                 sigma_r: float = 0.05, sigma_t: float = 0.1) -> PoseGraph:
    """Random directed multigraph without self-loops (ragged in/out degrees,
    repeated pairs allowed), ground truth poses uniform, random per-edge
    weights in [0.5, 2].  The last `isolated` vertices have no edges."""
    rng = np.random.default_rng(seed)
    q_gt = random_unit_quaternions(rng, n)
    t_gt = rng.uniform(-5.0, 5.0, (n, 3))
    live = max(n - isolated, 2)
    # skewed degrees: a few hubs
    w = rng.pareto(1.5, live) + 0.1
    w /= w.sum()
    src = rng.choice(live, size=m, p=w)
    dst = rng.integers(0, live - 1, size=m)
    dst = np.where(dst >= src, dst + 1, dst)
    wts = (rng.uniform(0.5, 2.0, m), rng.uniform(0.5, 2.0, m)) if weights else None
    return _finish("random", n, src, dst, q_gt, t_gt, rng, sigma_r, sigma_t, weights=wts)


def random_state(rng: np.random.Generator, n: int, scale_t: float = 5.0, scale_dual: float = 0.1):
    """A random ADMM state (p on S^3; q near p; t, s near each other; small
    multipliers) for one-step checks."""
    p = random_unit_quaternions(rng, n)
    q = p + 0.05 * rng.standard_normal((n, 4))
    t = rng.uniform(-scale_t, scale_t, (n, 3))
    s = t + 0.05 * rng.standard_normal((n, 3))
    lam = scale_dual * rng.standard_normal((n, 4))
    z = scale_dual * rng.standard_normal((n, 3))
    return {k: np.ascontiguousarray(v) for k, v in dict(p=p, q=q, t=t, s=s, lam=lam, z=z).items()}


def batch_graphs(count: int = 4096, n_min: int = 50, n_max: int = 20000, density=(0.5, 3.0),
                 sigma_r: float = 0.02, sigma_t: float = 0.1, seed: int = 4) -> list[PoseGraph]:
    """Independent random-walk graphs with n_g log-uniform in [n_min, n_max]
    and closure density ~ U(density) closures per pose within 3 m."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(n_min), math.log(n_max), count)).round().astype(int)
    dens = rng.uniform(density[0], density[1], count)
    seeds = rng.integers(0, 2 ** 62, count)
    return [random_walk_graph(int(ns[g]), n_closures=None, closure_density=float(dens[g]),
                              sigma_r=sigma_r, sigma_t=sigma_t, seed=int(seeds[g]), name=f"batch{g}")
            for g in range(count)]


# ---- the named workloads ----------------------------------------------------

def workload(name: str) -> PoseGraph:
    if name == "walk128":
        return random_walk_graph(128, n_closures=200, sigma_r=0.05, sigma_t=0.1, seed=1, name="walk128")
    if name == "helix25k":
        return helix_graph()
    if name == "lattice1m":
        return lattice_walk_graph()
    if name == "lattice1m_4m":
        # the same walk with closures at p = 0.57: 4,002,064 edges, the
        # "about 4M edges" of the 1M-pose lattice at the edge-to-pose ratio
        # the stated workload names
        return lattice_walk_graph(p_closure=0.57)
    if name == "walk10k":
        return random_walk_graph(10000, n_closures=20000, sigma_r=0.02, sigma_t=0.1, seed=5, name="walk10k")
    if name == "ring100":
        return ring_graph(100)
    if name == "ring5000":
        return ring_graph(5000)
    if name == "cube7":
        return cube_graph(7, 0.3)
    if name == "cube10":
        return cube_graph(10, 0.9)
    raise KeyError(name)
