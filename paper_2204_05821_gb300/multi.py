"""Several GPUs: one process per GPU, launched by torchrun.

Refinement of one graph does not shard here, so several GPUs run it as
independent replicas.  A batch of independent graphs shards with no
data-path collective: every rank refines the graphs assigned to it, and only
the host-side bookkeeping below (the assignment, the timing and the metrics)
uses torch.distributed.
"""
from __future__ import annotations

from typing import Dict, List, Sequence


def shard_graphs(edge_counts: Sequence[int], world: int) -> List[List[int]]:
    """Assign graphs to ranks, largest first to the least loaded rank, so
    every rank gets about the same number of edges.  Returns the graph
    indices of every rank, ascending."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(edge_counts)), key=lambda j: (-int(edge_counts[j]), j))
    load = [0] * world
    shards: List[List[int]] = [[] for _ in range(world)]
    for j in order:
        r = min(range(world), key=lambda q: (load[q], q))
        shards[r].append(j)
        load[r] += int(edge_counts[j])
    return [sorted(s) for s in shards]


def max_over_ranks(value: float) -> float:
    """The largest value over all ranks (the job's time is its slowest rank)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    backend = dist.get_backend()
    dev = "cuda" if backend == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_results(local: Dict[int, object]) -> Dict[int, object]:
    """Merge every rank's {graph index: result} on every rank."""
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return dict(local)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, local)
    merged: Dict[int, object] = {}
    for p in parts:
        merged.update(p)
    return merged
