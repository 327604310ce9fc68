"""The odometry start on the device against the oracle's.

The start composes the relative measurements along the spanning forest of
the earliest edges (an edge joins when it links two components, edges in
input order), each component rooted at its lowest vertex with the identity
pose.  The device (in pradmm_create) finds that forest by Boruvka's rounds
with the edge index as the weight and roots it by an Euler tour ranked by
pointer jumping; the start composes the poses by pointer jumping in segments;
the oracle scans the edges in order and walks each tree from its root.  The
forest (index work) is compared bit for bit, parent and tree-edge code of
every vertex; the poses within rounding.  The graphs below are chosen for the parts of the
device path the walk workloads leave easy: many Boruvka rounds (random edge
order), several components and isolated vertices, a chain whose hooks form
one long list (edges numbered against the chain, half of them reversed), a
hub whose tree hangs from a leaf, parallel and opposite edges, no edges at all.
Tolerance: FP64 on both sides, the same step formulas composed in another
association: 1e-11 on q, 1e-11 x (1 + max |t|) on t.
"""
import numpy as np
import pytest

import oracle
from paper_2601_15684_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2601_15684_gb300 import build_lib
    from paper_2601_15684_gb300 import pradmm
    build_lib.build()
    pradmm.load()
    return pradmm


def _graph(n, src, dst, seed):
    rng = np.random.default_rng(seed)
    q_gt = synth.random_unit_quaternions(rng, n)
    t_gt = rng.uniform(-20.0, 20.0, (n, 3))
    return synth._finish("odometry-case", n, np.asarray(src), np.asarray(dst), q_gt, t_gt, rng, 0.05, 0.1)


def _components(seed):
    # three random components on interleaved vertex ids (v mod 3), edges shuffled
    rng = np.random.default_rng(seed)
    n = 1500
    src, dst = [], []
    for c in range(3):
        ids = np.arange(c, n, 3)
        k = ids.size
        a = rng.integers(0, k, 3 * k)
        b = rng.integers(0, k - 1, 3 * k)
        b = np.where(b >= a, b + 1, b)
        src.append(ids[a])
        dst.append(ids[b])
    src, dst = np.concatenate(src), np.concatenate(dst)
    o = rng.permutation(src.size)
    return _graph(n, src[o], dst[o], seed)


def _reversed_chain(seed):
    # path 0 - 1 - ... - n-1, edge k joins n-2-k and n-1-k, every other edge reversed
    n = 4097
    k = np.arange(n - 1)
    a, b = n - 2 - k, n - 1 - k
    flip = (k % 2) == 1
    return _graph(n, np.where(flip, b, a), np.where(flip, a, b), seed)


def _hub(seed):
    # star around vertex 700 in random edge order, plus parallel and opposite edges
    rng = np.random.default_rng(seed)
    n = 1201
    leaves = np.setdiff1d(np.arange(n), [700])
    o = rng.permutation(leaves.size)
    src = np.full(leaves.size, 700)
    dst = leaves[o]
    dup = rng.choice(leaves, 200)
    src = np.concatenate([src, dup, np.full(200, 700)])
    dst = np.concatenate([dst, np.full(200, 700), dup])
    return _graph(n, src, dst, seed)


def _grid(seed):
    # 60 x 60 grid, edges in random order: Boruvka needs several rounds
    rng = np.random.default_rng(seed)
    s = 60
    v = np.arange(s * s).reshape(s, s)
    src = np.concatenate([v[:, :-1].ravel(), v[:-1, :].ravel()])
    dst = np.concatenate([v[:, 1:].ravel(), v[1:, :].ravel()])
    o = rng.permutation(src.size)
    return _graph(s * s, src[o], dst[o], seed)


CASES = {
    "random": lambda: synth.random_graph(3000, 9000, seed=1),
    "isolated": lambda: synth.random_graph(1200, 2500, seed=3, isolated=300),
    "components": lambda: _components(5),
    "reversed_chain": lambda: _reversed_chain(6),
    "hub": lambda: _hub(7),
    "grid": lambda: _grid(8),
    "two_vertices": lambda: _graph(2, [1], [0], 9),
    "no_edges": lambda: _graph(5, np.zeros(0, np.int64), np.zeros(0, np.int64), 10),
}


@pytest.mark.parametrize("case", list(CASES))
def test_device_odometry_matches_oracle(P, case):
    g = CASES[case]()
    q0, t0 = oracle.init_odometry(g)
    prm = P.pradmm_default_params()
    prm.precision = P.PRADMM_FP64
    with P.Solver(g, prm) as S:
        S.init_odometry()
        st = S.state()
    dq = float(np.abs(st["q"] - q0).max()) if g.n else 0.0
    dt = float(np.abs(st["t"] - t0).max()) if g.n else 0.0
    scale = 1.0 + float(np.abs(t0).max())
    print(f"{case}: n={g.n} m={g.m} max |dq| {dq:.2e}, max |dt| {dt:.2e} (|t| up to {scale - 1:.1f})")
    assert dq <= 1e-11, (case, dq)
    assert dt <= 1e-11 * scale, (case, dt)
    # the multipliers start at zero and s = t, p = q
    assert np.array_equal(st["p"], st["q"]) and np.array_equal(st["s"], st["t"])
    assert not np.any(st["lam"]) and not np.any(st["z"])


def test_device_odometry_repeated_and_after_steps(P):
    """A second start after iterations gives the same poses again (the
    composition's work space is rebuilt every call, the forest is create's)."""
    g = _components(11)
    q0, t0 = oracle.init_odometry(g)
    prm = P.pradmm_default_params()
    prm.precision = P.PRADMM_FP64
    with P.Solver(g, prm) as S:
        S.init_odometry()
        a = S.state()
        S.step(5)
        S.init_odometry()
        b = S.state()
    for k in ("q", "t"):
        assert np.array_equal(a[k], b[k]), k
    assert np.abs(a["q"] - q0).max() <= 1e-11


@pytest.mark.parametrize("case", list(CASES) + ["lattice1m"])
def test_device_forest_equals_oracle_forest(P, case):
    """The forest itself (index work) is compared bit for bit: every vertex's
    parent and tree-edge code from create's device forest against
    oracle.odometry_forest (pinned against brute force in
    tests/test_oracle_forest.py)."""
    g = synth.workload("lattice1m") if case == "lattice1m" else CASES[case]()
    par_o, pe_o = oracle.odometry_forest(g)
    with P.Solver(g) as S:
        par_d, pe_d = S.odometry_forest()
    bad = np.nonzero((par_d != par_o) | (pe_d != pe_o))[0]
    assert bad.size == 0, (case, bad[:10], par_d[bad[:10]], par_o[bad[:10]])
