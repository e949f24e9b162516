"""Multi-GPU host logic: objects are independent (each has its own MLP, rays,
optimiser and random stream, section 3.2), so a scene shards across ranks by
object with no collective on the data path. Only the timing and counts that
a job reports are reduced across ranks.

Results do not depend on the partition as long as every object keeps its
global random stream id (the Philox counter carries the stream id, not the
object's slot on a rank).
"""
import torch
import torch.distributed as dist


def object_cost(rays, samples_per_ray, hidden):
    """Work of one object per step, proportional to its MLP flops:
    rays x samples x (93 H + 3 H^2 + 4 H) multiply-adds, forward only (the
    backward is a fixed multiple of it)."""
    return rays * samples_per_ray * (93 * hidden + 3 * hidden * hidden + 4 * hidden)


def partition(costs, world):
    """Deterministic balanced split of objects over `world` ranks: largest
    cost first, each to the rank with the least load so far (ties to the
    lowest rank). Returns, per rank, its object indices in ascending order."""
    order = sorted(range(len(costs)), key=lambda k: (-costs[k], k))
    load = [0] * world
    out = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda i: (load[i], i))
        out[r].append(k)
        load[r] += costs[k]
    return [sorted(v) for v in out]


def _reduce(x, op):
    t = torch.tensor([float(x)], dtype=torch.float64)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        if dist.get_backend() == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x):
    """The job's time is its slowest rank's."""
    return _reduce(x, dist.ReduceOp.MAX)


def sum_over_ranks(x):
    """Units (samples, rays, steps) processed by the whole job."""
    return _reduce(x, dist.ReduceOp.SUM)
