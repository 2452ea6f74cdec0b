"""Host-side logic for running on N GPUs of one node (one process per GPU).

The single-problem path needs no data exchange between GPUs: every rank runs
its own replica of the workload (weak scaling), and independent instances of
a batch are split into contiguous shards, one per rank.  The only
collectives are timing bookkeeping: a barrier before and after the timed
region and the maximum of the per-rank times.  Works with the ``nccl``
backend on GPUs and with ``gloo`` on CPUs.
"""

from __future__ import annotations

import os


def env_ranks():
    """(world_size, rank, local_rank) from the launcher's environment (defaults: 1, 0, 0)."""
    def _i(name, d):
        try:
            return int(os.environ.get(name, d))
        except ValueError:
            return d
    return _i("WORLD_SIZE", 1), _i("RANK", 0), _i("LOCAL_RANK", 0)


def shard(n_items: int, rank: int, world: int):
    """Contiguous, balanced slice [start, stop) of n_items for this rank (sizes differ by at most 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    stop = start + base + (1 if rank < extra else 0)
    return start, stop


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def barrier():
    d = _dist()
    if d is not None:
        d.barrier()


def reduce_max(value: float) -> float:
    """Maximum of a per-rank float over all ranks (identity without a process group)."""
    d = _dist()
    if d is None:
        return float(value)
    import torch
    dev = "cuda" if d.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    d.all_reduce(t, op=d.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float) -> float:
    d = _dist()
    if d is None:
        return float(value)
    import torch
    dev = "cuda" if d.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    d.all_reduce(t, op=d.ReduceOp.SUM)
    return float(t.item())
