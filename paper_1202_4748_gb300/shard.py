"""Ensemble sharding across ranks (one process per GPU).

The systems of an ensemble are independent and their noise is keyed by
(site, step, system_id), so a system's trajectory does not depend on which
rank advances it: the only exchange is a final gather of the FP64
accumulators (a few hundred bytes per system).  ``partition`` balances site
counts with a greedy largest-first bin packing; ``gather`` collects per-system
results in descriptor order on every rank through torch.distributed (any
backend that supports object collectives, e.g. gloo on CPU or nccl on GPU).
"""


def partition(systems, world):
    """List, per rank, of the indices of the systems that rank advances."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(systems)),
                   key=lambda k: (-systems[k]["nx"] * systems[k]["ny"] * systems[k]["nz"], k))
    load = [0] * world
    out = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda i: (load[i], i))
        out[r].append(k)
        load[r] += systems[k]["nx"] * systems[k]["ny"] * systems[k]["nz"]
    return [sorted(x) for x in out]


def gather(local, n_systems, group=None):
    """Merge {system index: result} dicts from all ranks into a list in system order."""
    import torch.distributed as dist
    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, local, group=group)
    merged = {}
    for p in parts:
        for k, v in p.items():
            if k in merged:
                raise RuntimeError("system %d advanced by two ranks" % k)
            merged[k] = v
    if sorted(merged) != list(range(n_systems)):
        raise RuntimeError("missing systems after gather")
    return [merged[k] for k in range(n_systems)]
