"""Multi-process host logic (gloo, world size 2, CPU): the timing reductions
bench.py uses under torchrun, the weak-scaling seeds, the LPT split, and a
fixed channel set split over two ranks end to end -- each rank decomposes its
share (the CPU oracle stands in for the GPU path) and rank 0 gathers the
per-channel records."""
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


def _split_worker(rank, world, port, q, sizes, tol, l):
    import numpy as np
    import torch.distributed as dist

    from oracle import rsvd as orsvd
    from paper_2307_15572_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        parts = shard.split_channels(sizes, l, 0, world)
        recs = []
        for c in parts[rank]:
            A = synth.batch_channel(c, sizes[c], seed=77)
            r = orsvd.rsvd(A, tol=tol, l=l, q=0, seed=5)
            err = orsvd.reconstruct_error(A, r.U, r.S, r.V)
            recs.append({"index": c, "rank_of": rank, "k": r.k, "err": err, "status": 0})
        got = shard.gather_records(dist, recs)
        tot, mx = shard.reduce_timing(dist, float(sum(sizes[c] ** 2 for c in parts[rank])), 1.0 + rank)
        q.put((rank, got, parts, tot, mx))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_fixed_set_split_and_gather_two_ranks():
    import torch.multiprocessing as mp

    from oracle import rsvd as orsvd
    from paper_2307_15572_gb300 import synth
    sizes = [300, 120, 260, 90, 200, 150, 310]
    tol, l = 1e-3, 40
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_worker, args=(r, 2, port, q, sizes, tol, l)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, got0, parts0, tot0, mx0), (r1, got1, parts1, tot1, mx1) = res
    assert got1 is None and parts0 == parts1                     # same split on every rank
    assert sorted(parts0[0] + parts0[1]) == list(range(len(sizes)))
    assert [g["index"] for g in got0] == list(range(len(sizes)))  # every channel once, in order
    assert {g["rank_of"] for g in got0 if g["index"] in parts0[1]} == {1}
    assert tot0 == tot1 == float(sum(n * n for n in sizes)) and mx0 == mx1 == 2.0
    # the gathered records are the single-process results
    for g in got0:
        c = g["index"]
        A = synth.batch_channel(c, sizes[c], seed=77)
        r = orsvd.rsvd(A, tol=tol, l=l, q=0, seed=5)
        assert g["k"] == r.k and abs(g["err"] - orsvd.reconstruct_error(A, r.U, r.S, r.V)) <= 1e-15


def test_split_balances_channel_work():
    sizes = [12000, 11000, 3000, 2500, 9000, 1000, 4000, 8000]
    parts = shard.split_channels(sizes, 128, 0, 3)
    costs = shard.channel_costs(sizes, 128, 0)
    loads = sorted(sum(costs[i] for i in p) for p in parts)
    assert sorted(i for p in parts for i in p) == list(range(len(sizes)))
    assert loads[-1] <= (4 / 3 - 1 / 9) * max(max(costs), sum(costs) / 3)
