"""Multi-process host logic (gloo, world size 2, CPU): the timing reductions
bench.py uses under torchrun, the weak-scaling seeds and the LPT split."""
import os
import socket

import pytest

from paper_2307_15572_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r decomposed (r + 1) * 1e9 entries in 10 (r + 1) ms
        tot, mx = shard.reduce_timing(dist, (rank + 1) * 1e9, 10.0 * (rank + 1))
        q.put((rank, tot, mx, shard.rank_seed(15572002, rank)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_timing_reduction_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tot, mx, seed in res:
        assert tot == 3e9 and mx == 20.0        # whole-job entries, slowest rank's time
    assert res[0][3] != res[1][3]               # weak scaling: different channel sets


def test_single_process_reduction_is_identity():
    assert shard.reduce_timing(None, 5.0, 7.0) == (5.0, 7.0)


def test_lpt_balances_and_covers():
    costs = [9, 7, 6, 5, 4, 3, 3, 2]
    parts = shard.lpt(costs, 3)
    assert sorted(i for p in parts for i in p) == list(range(len(costs)))
    loads = [sum(costs[i] for i in p) for p in parts]
    # LPT guarantee: makespan <= (4/3 - 1/(3m)) OPT; here OPT = 13
    assert max(loads) <= (4 / 3 - 1 / 9) * 13
    assert shard.lpt([1.0], 4) == [[0], [], [], []]
