"""Pins of the oracle's odometry forest (oracle.odometry_forest), the index
work behind the odometry start, against brute force on small graphs.

The start composes the measurements along the forest in which an edge joins
when it links two components, edges taken in input order, each component
rooted at its lowest vertex.  Checked here without reusing that procedure:
- an edge is in the forest exactly when its endpoints are not yet joined by
  the edges before it (breadth-first reachability over the earlier edges);
- the roots are exactly the lowest vertex of every connected component;
- each non-root vertex's code names a forest edge joining it to its parent,
  e when it is the edge's head and -(e + 2) when it is its tail;
- following parents from any vertex reaches its component's root.
Given the forest and the roots the parents are unique, so these fix the
output completely.
"""
from collections import deque

import numpy as np
import pytest

import oracle
from paper_2601_15684_gb300 import synth


def _reachable(n, src, dst, upto, a, b):
    adj = [[] for _ in range(n)]
    for e in range(upto):
        adj[src[e]].append(dst[e])
        adj[dst[e]].append(src[e])
    seen = {a}
    dq = deque([a])
    while dq:
        v = dq.popleft()
        if v == b:
            return True
        for w in adj[v]:
            if w not in seen:
                seen.add(w)
                dq.append(w)
    return False


def _components(n, src, dst):
    adj = [[] for _ in range(n)]
    for a, b in zip(src, dst):
        adj[a].append(b)
        adj[b].append(a)
    comp = [-1] * n
    for r in range(n):
        if comp[r] >= 0:
            continue
        comp[r] = r
        dq = deque([r])
        while dq:
            v = dq.popleft()
            for w in adj[v]:
                if comp[w] < 0:
                    comp[w] = r
                    dq.append(w)
    return comp


def _graph(n, src, dst, seed):
    rng = np.random.default_rng(seed)
    q = synth.random_unit_quaternions(rng, n)
    t = rng.uniform(-5, 5, (n, 3))
    return synth._finish("forest-case", n, np.asarray(src), np.asarray(dst), q, t, rng, 0.05, 0.1)


def _cases():
    rng = np.random.default_rng(7)
    out = []
    for k in range(12):
        n = int(rng.integers(2, 45))
        m = int(rng.integers(0, 3 * n))
        a = rng.integers(0, n, m)
        b = rng.integers(0, n - 1, m)
        b = np.where(b >= a, b + 1, b)  # no self-loops
        if k % 3 == 0 and m:
            a, b = np.concatenate([a, b[:4]]), np.concatenate([b, a[:4]])  # opposite parallel edges
        out.append(_graph(n, a, b, k))
    n = 30  # a chain whose edges run against the vertex order, half of them reversed
    e = np.arange(n - 1)
    x, y = n - 2 - e, n - 1 - e
    out.append(_graph(n, np.where(e % 2 == 1, y, x), np.where(e % 2 == 1, x, y), 99))
    out.append(_graph(6, np.zeros(0, np.int64), np.zeros(0, np.int64), 100))  # no edges
    return out


@pytest.mark.parametrize("g", _cases(), ids=lambda g: f"n{g.n}_m{g.m}")
def test_odometry_forest_against_brute_force(g):
    par, pedge = oracle.odometry_forest(g)
    n, src, dst = g.n, [int(x) for x in g.src], [int(x) for x in g.dst]
    # the forest edges named by the codes
    used = set()
    for v in range(n):
        c = int(pedge[v])
        if par[v] < 0:
            assert c == -1, (v, c)
            continue
        if c >= 0:
            e = c
            assert dst[e] == v and src[e] == par[v], (v, c)
        else:
            e = -c - 2
            assert src[e] == v and dst[e] == par[v], (v, c)
        assert e not in used, e
        used.add(e)
    # Kruskal by edge order, by reachability over the earlier edges
    expect = {e for e in range(g.m) if not _reachable(n, src, dst, e, src[e], dst[e])}
    assert used == expect
    # roots: the lowest vertex of each component; parents lead there
    comp = _components(n, src, dst)
    roots = {v for v in range(n) if par[v] < 0}
    assert roots == set(comp)
    assert all(comp[r] == r for r in roots)
    for v in range(n):
        x, steps = v, 0
        while par[x] >= 0:
            x = int(par[x])
            steps += 1
            assert steps <= n
        assert x == comp[v]


def test_odometry_forest_matches_the_walk_of_init_odometry():
    # the poses of init_odometry follow the forest: each non-root pose is its
    # parent's composed with the tree edge's measurement (or its inverse)
    g = synth.random_graph(300, 900, seed=21, isolated=10)
    par, pedge = oracle.odometry_forest(g)
    q, t = oracle.init_odometry(g)
    for v in range(g.n):
        if par[v] < 0:
            np.testing.assert_array_equal(q[v], [1.0, 0.0, 0.0, 0.0])
            np.testing.assert_array_equal(t[v], [0.0, 0.0, 0.0])
            continue
        p = int(par[v])
        c = int(pedge[v])
        e = c if c >= 0 else -c - 2
        qe, te = g.q_meas[e] / np.linalg.norm(g.q_meas[e]), g.t_meas[e]
        if c >= 0:  # parent -> v along the edge
            qv = synth._qmul(q[p], qe)
            tv = t[p] + synth._rotate(q[p], te)
        else:  # v -> parent: the inverse step
            qv = synth._qmul(q[p], synth._qconj(qe))
            tv = t[p] - synth._rotate(qv, te)
        np.testing.assert_allclose(q[v], qv, atol=1e-12)
        np.testing.assert_allclose(t[v], tv, atol=1e-9)
