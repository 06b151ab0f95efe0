"""Host-side logic of the multi-GPU (one process per GPU) runs.

Channels are independent problems, so GPUs share no data: weak scaling gives
every rank its own seeded channel set; a fixed set is split by longest
processing time first (LPT) on the cost n^2 l (2q + 2) of a channel.  The only
collectives are the timing reductions below (max of the step time, sum of the
entries) and the gather of per-channel result records (status, rank, error,
time) to rank 0 -- host metadata, never the data path.
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


def channel_costs(sizes, l, q):
    """Work of each channel: its passes over V, n^2 l (2q + 2)."""
    return [float(n) * n * l * (2 * q + 2) for n in sizes]


def split_channels(sizes, l, q, nranks):
    """LPT split of a fixed channel set over nranks ranks (index lists)."""
    return lpt(channel_costs(sizes, l, q), nranks)


def gather_records(dist, records, dst=0):
    """Per-channel result records (dicts with an "index" key) of every rank,
    merged and sorted by index on rank dst (None on the other ranks); the
    local list itself without dist."""
    if dist is None:
        return sorted(records, key=lambda r: r["index"])
    out = [None] * dist.get_world_size() if dist.get_rank() == dst else None
    dist.gather_object(list(records), out, dst=dst)
    if out is None:
        return None
    return sorted((r for part in out for r in part), key=lambda r: r["index"])
