"""Several GPUs of one node as independent replicas.

The rays of the method are independent (Sec. 2): there is no exchange on the
data path, so N GPUs run N processes (one per GPU, launched by torchrun), each
with its own context and state buffers.  A replica either traces its own copy
of a workload (weak scaling, the benchmark) or its share of a list of work
items (images, requests) routed to it by the host.  The only collectives are
host-side: a barrier around a timed region and the maximum of the ranks'
elapsed times.
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass
class Rank:
    rank: int = 0
    world: int = 1
    local: int = 0


def from_env() -> Rank:
    """RANK / WORLD_SIZE / LOCAL_RANK as torchrun sets them (1 process if unset)."""
    return Rank(int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
                int(os.environ.get("LOCAL_RANK", "0")))


def init(r: Rank, backend: str):
    """Join the process group when there is more than one rank; returns the
    torch.distributed module or None."""
    if r.world <= 1:
        return None
    import torch
    import torch.distributed as dist
    if backend == "nccl":
        torch.cuda.set_device(r.local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", r.local))
    else:
        dist.init_process_group(backend)
    return dist


def max_over_ranks(dist, value: float, device="cpu") -> float:
    """The largest of the ranks' values (a rank's elapsed time, say)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, max_ms: float, world: int) -> float:
    """Whole-job throughput of `world` replicas that each processed
    units_per_rank units, the slowest in max_ms milliseconds."""
    return world * units_per_rank / (max_ms / 1000.0)


def shard(n: int, rank: int, world: int):
    """Contiguous share (first, count) of n work items for `rank`: the first
    n % world ranks take one item more."""
    base, extra = divmod(int(n), int(world))
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def route(items, rank: int, world: int):
    """Items of a stream (requests, images) served by `rank`: round robin on
    their position, so arrivals spread evenly over the replicas."""
    return [x for k, x in enumerate(items) if k % world == rank]


__all__ = ["Rank", "from_env", "init", "max_over_ranks", "job_rate", "shard", "route"]
