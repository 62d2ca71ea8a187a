"""Replica runs on the GPUs of one node.

The training step and the ray march shard by points and pixels with no
exchange the method needs (Sec. 4 trains one network on one GPU), so a run on
N GPUs is N independent replicas, one process per GPU: each rank trains its own
network on its own points.  The ranks meet only at a barrier around the timed
region and in a max-reduction of the timed interval; the whole-job throughput
is the units all ranks processed over the slowest rank's time.  There is no
data-path collective.
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
