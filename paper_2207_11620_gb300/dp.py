"""Data-parallel training step: one network replicated over the ranks of a
torch.distributed process group (one GPU each), each rank training on a
disjoint shard of the global batch, one exchange of the gradient per step.

Sec. 4 trains one network per volume on one GPU; its training step is a sum
over the batch's points (the mean loss and its gradient), so the points split
across GPUs with one reduction of the gradient:

  rank r   nv_train_grad on its shard: the gradient of the GLOBAL mean loss is
           added into its gradient buffer, its shard's loss sum is written
  all      all-reduce (sum) of the gradient buffers and of the loss sums,
           all-reduce (max) of the two step flags (an FP16 overflow: every rank
           skips the step; a point outside [0,1]^3: every rank leaves the
           reachable-block skipping of Adam alike)
  rank r   nv_optimizer_step: the same update of the same parameters on every
           rank, so the replicas stay identical

Host-side orchestration only: the arithmetic runs in the library's kernels.  A
replica is any object with train_grad(xyz, target, n_total) -> loss sum,
dp_buffers() -> (gradient, flags) and optimizer_step() -- NeuralVolume on a
GPU.

Rendering splits by image rows (render_tiles): Sec. 5.2.1 marches and
composites each pixel's ray on its own, so every rank renders its band of rows
(nv_render_rows) with no exchange, and the bands are gathered only to assemble
the frame.
"""
from __future__ import annotations


def shard(n_total: int, rank: int, world: int) -> tuple[int, int]:
    """[lo, hi) of rank's contiguous shard: the first n_total % world ranks take
    one point more; the shards are disjoint and cover [0, n_total)."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError(f"shard: n_total={n_total}, rank={rank}, world={world}")
    base, extra = divmod(n_total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


class DataParallelStep:
    """One training step of a replica over its shard, the reductions, the update.

    group: a torch.distributed process group (None: the default group when one
    is initialised, else a single rank with nothing to reduce)."""

    def __init__(self, replica, group=None):
        import torch.distributed as dist
        self.replica = replica
        self.group = group
        self.dist = dist if dist.is_available() and dist.is_initialized() else None
        self.world = self.dist.get_world_size(group) if self.dist else 1
        self.rank = self.dist.get_rank(group) if self.dist else 0

    def step_shard(self, xyz, target, n_total: int):
        """This rank's shard (xyz [n][3], target [n]) of a global batch of n_total
        points; returns the global mean loss (a one-element tensor, every rank)."""
        loss_sum = self.replica.train_grad(xyz, target, n_total)
        grads, flags = self.replica.dp_buffers()
        if self.world > 1:
            d = self.dist
            d.all_reduce(grads, op=d.ReduceOp.SUM, group=self.group)
            d.all_reduce(flags, op=d.ReduceOp.MAX, group=self.group)
            d.all_reduce(loss_sum, op=d.ReduceOp.SUM, group=self.group)
        self.replica.optimizer_step()
        return loss_sum / n_total

    def __call__(self, xyz, target):
        """The whole global batch (the same on every rank): this rank takes its shard."""
        n_total = xyz.shape[0]
        lo, hi = shard(n_total, self.rank, self.world)
        return self.step_shard(xyz[lo:hi], target[lo:hi], n_total)


def render_tiles(render_band, width: int, height: int, group=None):
    """One frame split into row bands over the ranks of `group` (None: the
    default group when one is initialised, else one rank renders everything).

    render_band(row0, rows) renders rows [row0, row0 + rows) of the image and
    returns them as a tensor [rows][width][4] (e.g. Renderer.render(..., rows=
    (row0, rows))).  Rank r takes the rows shard(height, r, world); the bands
    are all-gathered (padded to the largest band) so every rank returns the
    whole image [height][width][4] on the device of its band."""
    import torch
    import torch.distributed as dist
    d = dist if dist.is_available() and dist.is_initialized() else None
    world = d.get_world_size(group) if d else 1
    rank = d.get_rank(group) if d else 0
    lo, hi = shard(height, rank, world)
    band = render_band(lo, hi - lo) if hi > lo else None
    if world == 1:
        return band
    most = -(-height // world)
    dev = band.device if band is not None else ("cuda" if d.get_backend(group) == "nccl" else "cpu")
    dtype = band.dtype if band is not None else torch.float32
    buf = torch.zeros((most, width, 4), dtype=dtype, device=dev)
    if band is not None:
        if tuple(band.shape) != (hi - lo, width, 4):
            raise ValueError(f"render_band({lo}, {hi - lo}) returned {tuple(band.shape)}")
        buf[: hi - lo] = band
    parts = [torch.empty_like(buf) for _ in range(world)]
    d.all_gather(parts, buf, group=group)
    rows = [shard(height, r, world) for r in range(world)]
    return torch.cat([parts[r][: b - a] for r, (a, b) in enumerate(rows)], dim=0)
