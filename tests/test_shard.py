"""Multi-rank host logic on CPU (gloo, world_size 2): the by-graph split of the
batched form and the max / sum reductions the benchmark uses.  No GPU."""
import os
import socket

import numpy as np
import pytest

from paper_2601_15684_gb300.shard import shard_graphs


def test_shard_is_a_balanced_partition():
    rng = np.random.default_rng(0)
    sizes = np.exp(rng.uniform(np.log(50), np.log(20000), 4096)).astype(int) * 3
    for world in (1, 2, 3, 8):
        parts = shard_graphs(sizes, world)
        allg = np.concatenate(parts)
        assert np.array_equal(np.sort(allg), np.arange(sizes.size))  # disjoint and complete
        loads = np.array([sizes[p].sum() for p in parts])
        # LPT bound: max load <= mean + largest item
        assert loads.max() <= loads.mean() + sizes.max()
        assert shard_graphs(sizes, world)[0].tolist() == parts[0].tolist()  # deterministic


def test_shard_small_cases():
    assert [p.tolist() for p in shard_graphs([5, 1, 1, 1, 1, 1], 2)] == [[0], [1, 2, 3, 4, 5]]
    assert [p.tolist() for p in shard_graphs([], 3)] == [[], [], []]
    with pytest.raises(ValueError):
        shard_graphs([1], 0)


def _worker(rank, world, port, sizes, out):
    import torch.distributed as dist

    from paper_2601_15684_gb300.shard import max_over_ranks, shard_graphs, sum_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard_graphs(sizes, world)[rank]
    work = float(np.asarray(sizes)[mine].sum())
    t_max = max_over_ranks(1.0 + rank)        # the slowest rank's time
    total = sum_over_ranks(work)              # work done by all ranks
    count = sum_over_ranks(len(mine))
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, mine.tolist(), t_max, total, count))


def test_gloo_world_size_two():
    import multiprocessing as mp

    sizes = [900, 10, 500, 400, 30, 70, 250]
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, g0, m0, s0, c0), (r1, g1, m1, s1, c1) = res
    assert sorted(g0 + g1) == list(range(len(sizes))) and not set(g0) & set(g1)
    assert m0 == m1 == 2.0
    assert s0 == s1 == float(sum(sizes))
    assert c0 == c1 == len(sizes)
