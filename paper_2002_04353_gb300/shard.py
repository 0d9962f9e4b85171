"""Host-side sharding of independent cases over the ranks of a job.

One process per GPU; the cases of a sweep are independent problems, so the
data path needs no exchange: each rank steps its own cases, and only the
timing and the node count are reduced at the end (the maximum time over the
ranks, the sum of the nodes).
"""


def assign_cases(node_counts, world):
    """Case indices per rank, balancing node counts greedily: cases taken
    largest first, each to the rank with the fewest nodes so far (the lower
    rank on ties).  Every case goes to exactly one rank; each rank's list is
    in increasing case order.  The largest rank load exceeds the mean by less
    than the largest case."""
    if world < 1:
        raise ValueError("world must be at least 1")
    load = [0] * world
    shards = [[] for _ in range(world)]
    order = sorted(range(len(node_counts)), key=lambda c: (-node_counts[c], c))
    for c in order:
        r = min(range(world), key=lambda k: (load[k], k))
        shards[r].append(c)
        load[r] += node_counts[c]
    return [sorted(s) for s in shards]


def max_over_ranks(value, torch, device=None):
    """The largest value over the ranks of the default process group (the
    value itself without one)."""
    dist = torch.distributed
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def sum_over_ranks(value, torch, device=None):
    """The sum of value over the ranks of the default process group."""
    dist = torch.distributed
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t)
    return float(t[0])
