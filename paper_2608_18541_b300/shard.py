"""Sharding of independent instances over ranks (one process per GPU).

Instances never exchange data (the paper's task-level replicas, Sec. II.F),
so a multi-GPU run needs no collective on the data path: each rank builds a
system from its own subset of instances with instance_base / global ids so
that the noise streams, keyed by the global instance id, are the same as in
a single-GPU run.  Only timings and results are gathered on the host.
"""


def contiguous_shards(costs, world):
    """Split instances 0..n-1 into `world` contiguous ranges of nearly equal
    total cost (e.g. atoms x steps).  Contiguous ranges keep each rank's
    global ids base, base+1, ..., which is how a system keys its noise
    (instance_base + local index).  Returns [(base, count)] per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    n = len(costs)
    total = float(sum(costs))
    out, start, acc = [], 0, 0.0
    for r in range(world):
        if r == world - 1:
            end = n
        else:
            target = total * (r + 1) / world
            end = start
            # take at least one instance while every later rank can still
            # get one, then extend while the running sum stays closer to the
            # target
            while end < n - (world - 1 - r) and (end == start or acc + costs[end] - target <= target - acc):
                acc += costs[end]
                end += 1
        out.append((start, end - start))
        start = end
    return out


def weak_shard(n_local, rank):
    """Weak scaling: every rank runs n_local instances of its own, with
    global ids rank * n_local ... rank * n_local + n_local - 1."""
    return rank * n_local, n_local


def subset(sysd, ids):
    """System description holding only the given instances (global ids)."""
    inst = sysd.get("instances")
    if not inst:
        raise ValueError("the description has no instance list")
    out = dict(sysd)
    out["instances"] = [inst[i] for i in ids]
    return out
