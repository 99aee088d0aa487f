"""Replica parallelism over independent problems: the instances of a sweep or
a request stream are split across ranks (one GPU each) with nothing
exchanged on the data path; ranks only agree on timing at the end.  Host
logic only, usable with any torch.distributed backend (gloo on CPU in the
tests, NCCL on GPUs)."""
from __future__ import annotations


def partition(costs, world):
    """Longest-processing-time split of instances with the given cost
    estimates over `world` ranks: instances in decreasing cost, each to the
    least-loaded rank (ties to the lower rank), so every rank gets a share of
    nearly equal total cost.  Deterministic; returns one sorted index list per
    rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def my_share(costs, rank, world):
    return partition(costs, world)[rank]


def max_over_ranks(value):
    """Largest value over all ranks (the job's time is its slowest rank's);
    the value itself without an initialised process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value):
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
