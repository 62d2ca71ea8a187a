"""Process-group plumbing of a run on the GPUs of one node (one process per GPU).

The ranks join a process group, meet at a barrier around the timed region and
take the max of their timed intervals; the whole-job throughput is the units
all ranks processed over the slowest rank's time.  The training step itself is
data parallel (dp.py): one network replicated on every rank, each rank on its
own shard of the global batch, one all-reduce of the gradient per step.
"""
from __future__ import annotations

import os


def setup(backend: str | None = None):
    """(world size, rank, local rank) from the launcher's environment; joins the
    process group when there is more than one rank (NCCL with CUDA, else gloo)."""
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cuda = torch.cuda.is_available() and backend != "gloo"
    if cuda:
        torch.cuda.set_device(local if ws > 1 else 0)
    if ws > 1:
        import torch.distributed as dist
        if cuda:
            dist.init_process_group(backend or "nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend or "gloo")
    return ws, rank, local


def barrier(ws: int) -> None:
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws: int, v: float) -> float:
    """The largest v over all ranks (every rank gets it)."""
    if ws == 1:
        return float(v)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ws: int, units_per_rank: float, seconds_max: float) -> float:
    """Whole-job rate: the units of every rank over the slowest rank's time."""
    return ws * units_per_rank / seconds_max


def teardown(ws: int) -> None:
    if ws > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()
