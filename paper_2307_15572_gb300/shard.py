"""Host-side logic of the multi-GPU (one process per GPU) runs.

Channels are independent problems, so GPUs share no data: weak scaling gives
every rank its own seeded channel set; a fixed set is split by longest
processing time first (LPT) on the cost n^2 l (2q + 2) of a channel.  The only
collectives are the timing reductions below (max of the step time, sum of the
entries), never on the data path.
"""

import heapq


def rank_seed(base_seed, rank):
    """Seed of rank `rank`'s channel set under weak scaling."""
    return int(base_seed) + int(rank)


def lpt(costs, nranks):
    """Assign items (by cost) to nranks bins, largest first onto the lightest bin.

    Returns a list of index lists; ties between bins go to the lower rank."""
    bins = [(0.0, r) for r in range(nranks)]
    heapq.heapify(bins)
    out = [[] for _ in range(nranks)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        load, r = heapq.heappop(bins)
        out[r].append(i)
        heapq.heappush(bins, (load + costs[i], r))
    return out


def reduce_timing(dist, entries, ms, device="cpu"):
    """(sum of entries over ranks, max of ms over ranks); identity without dist."""
    if dist is None:
        return float(entries), float(ms)
    import torch
    t = torch.tensor([float(entries)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    m = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return float(t.item()), float(m.item())
