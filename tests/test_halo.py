"""The vertex-partitioned plain iteration (paper_2601_15684_gb300/halo.py) on
CPU ranks (gloo): a graph split in walk order across 2 and 3 ranks, each rank
running the oracle's blocks on its local graph with the three halo exchanges
between them, gives every owned vertex bitwise the state of the single-rank
oracle iteration, and the all-reduced residual to rounding.  No GPU."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2601_15684_gb300 import halo, synth

KEYS = ("p", "q", "t", "s", "lam", "z")


def _graph():
    # a walk whose closures join poses far apart in walk order: many cut edges
    return synth.random_walk_graph(1500, n_closures=2500, sigma_r=0.05, sigma_t=0.1, seed=21)


def test_partition_is_contiguous_and_balanced():
    g = _graph()
    for world in (1, 2, 3, 5):
        rg = halo.partition(g.n, g.src, g.dst, world)
        assert rg[0][0] == 0 and rg[-1][1] == g.n
        assert all(rg[r][1] == rg[r + 1][0] for r in range(world - 1))
        w = 1 + np.bincount(g.src, minlength=g.n) + np.bincount(g.dst, minlength=g.n)
        loads = np.array([w[lo:hi].sum() for lo, hi in rg])
        assert loads.max() <= w.sum() / world + w.max()
    with pytest.raises(ValueError):
        halo.partition(10, [], [], 0)


@pytest.mark.parametrize("world", [2, 3, 4])
def test_plans_agree_across_ranks(world):
    g = _graph()
    rg = halo.partition(g.n, g.src, g.dst, world)
    plans = [halo.HaloPlan(g.n, g.src, g.dst, rg, r) for r in range(world)]
    for r, pr in enumerate(plans):
        lo, hi = rg[r]
        assert np.array_equal(pr.verts[:hi - lo], np.arange(lo, hi))
        # every edge with an endpoint owned by r is local to r, in input order
        e = np.nonzero(((g.src >= lo) & (g.src < hi)) | ((g.dst >= lo) & (g.dst < hi)))[0]
        assert np.array_equal(pr.edges, e)
        assert np.array_equal(pr.verts[pr.src], g.src[e]) and np.array_equal(pr.verts[pr.dst], g.dst[e])
        for kind in halo.KINDS:
            for peer, ids in pr.send[kind].items():
                got = plans[peer].verts[plans[peer].recv[kind][r]]
                assert np.array_equal(pr.verts[ids], got), (r, peer, kind)
                assert ((pr.verts[ids] >= lo) & (pr.verts[ids] < hi)).all()
            # every ghost of this kind is received from its owner exactly once
            recv = np.concatenate([pr.verts[v] for v in pr.recv[kind].values()] or [np.zeros(0, np.int64)])
            assert recv.size == np.unique(recv).size
    # a single rank has nothing to exchange
    one = halo.HaloPlan(g.n, g.src, g.dst, [(0, g.n)], 0)
    assert all(not one.send[k] and not one.recv[k] for k in halo.KINDS) and one.n_local == g.n


def _worker(rank, world, port, iters, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = _graph()
        q0, t0 = oracle.init_odometry(g)
        st_full = oracle.init_state(q0, t0)
        rg = halo.partition(g.n, g.src, g.dst, world)
        plan = halo.HaloPlan(g.n, g.src, g.dst, rg, rank)
        lg = synth.PoseGraph(n=plan.n_local, src=plan.src, dst=plan.dst, q_meas=g.q_meas[plan.edges],
                             t_meas=g.t_meas[plan.edges], kappa=g.kappa[plan.edges], omega=g.omega[plan.edges])
        prm = oracle.make_params(beta1=1.0, beta2=1.0, tau=1.5)
        c = np.zeros((lg.m, 3))
        st = plan.local_rows(st_full)
        es = []
        for _ in range(iters):
            es.append(halo.iterate_partitioned(plan, lambda w, x: oracle.block(lg, prm, x, w, c), st, (1.0, 1.0)))
        owned = {k: st[k][:plan.n_owned] for k in KEYS}
        out.put((rank, rg[rank], owned, es, plan.halo_bytes()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_partitioned_iteration_equals_single_rank_oracle(world):
    import multiprocessing as mp

    iters = 6
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, iters, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = _graph()
    q0, t0 = oracle.init_odometry(g)
    st = oracle.init_state(q0, t0)
    prm = oracle.make_params(beta1=1.0, beta2=1.0, tau=1.5)
    es = []
    for _ in range(iters):
        st, r, _ = oracle.iterate(g, prm, st, 1)
        es.append(r[0])
    for rank, (lo, hi), owned, e_part, hb in res:
        for k in KEYS:
            np.testing.assert_array_equal(owned[k], st[k][lo:hi], err_msg=f"rank {rank} {k}")
        np.testing.assert_allclose(e_part, es, rtol=1e-12)
        assert sum(hb.values()) > 0  # the split cuts edges: there is a halo
