"""The data-parallel training step (paper_2207_11620_gb300/dp.py) on the CPU:
two gloo ranks, each a replica whose arithmetic is the FP64 oracle, train on
the two halves of a global batch; the result must equal one rank training on
the whole batch (Sec. 4's step: the loss is a mean over the batch, its gradient
a sum), and the replicas must stay identical.  The oracle is the checker here:
the library's own replica (NeuralVolume) runs the same orchestration on GPUs
(tests/test_gpu_dp.py checks its kernels' side on one GPU)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2207_11620_gb300 import dp  # noqa: E402

LR = 1e-2


class OracleReplica:
    """A replica whose training arithmetic is the oracle's (L2 loss, Adam)."""

    def __init__(self, net, params):
        import oracle as O
        self.O, self.net = O, net
        self.p = np.asarray(params, np.float64).copy()
        self.m = np.zeros_like(self.p)
        self.v = np.zeros_like(self.p)
        self.t = 0
        self.g = torch.zeros(net.n_params, dtype=torch.float64)
        self.flags = torch.zeros(2, dtype=torch.int32)  # (overflow, off-domain)

    def train_grad(self, xyz, target, n_total):
        x, t = xyz.numpy(), target.numpy()
        if x.shape[0] == 0:
            return torch.zeros(1, dtype=torch.float64)
        y = self.O.forward(self.net, self.p, x)
        r = y - t.astype(np.float64)
        self.g += torch.from_numpy(self.O.backward(self.net, self.p, x, 2.0 * r / n_total))
        return torch.tensor([float(np.sum(r * r))], dtype=torch.float64)

    def dp_buffers(self):
        return self.g, self.flags

    def optimizer_step(self):
        if self.flags[0] == 0:
            self.t += 1
            self.O.adam(self.p, self.g.numpy(), self.m, self.v, self.t, lr=LR)
        self.flags[0] = 0
        self.g.zero_()


def _problem():
    import oracle as O
    from paper_2207_11620_gb300 import inputs as I
    net = O.Net(L=4, F=2, log2T=10, Nmin=4, b=1.6, dims=(8, 16, 16, 1))
    params = I.init_params(net.n_table, net.n_weights, seed=3, table_scale=0.1, dims=net.dims)
    vol = I.blob_volume(16, seed=2)
    batches = []
    for s in range(3):
        x = O.sample_points(5, s, 0, 1001)  # odd: the shards differ by one point
        batches.append((x, O.trilinear(vol, x).astype(np.float32)))
    return net, params, batches


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, ws, port, q, overflow_rank):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    net, params, batches = _problem()
    rep = OracleReplica(net, params)
    step = dp.DataParallelStep(rep)
    losses = []
    for i, (x, t) in enumerate(batches):
        if i == 1 and rank == overflow_rank:
            rep.flags[0] = 1  # this rank's backward overflowed: every rank must skip
        losses.append(float(step(torch.from_numpy(x), torch.from_numpy(t))[0]))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, rep.p, rep.t, losses))


def _run(ws, overflow_rank=-1):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q, overflow_rank)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in range(ws)), key=lambda o: o[0])
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    return out


def test_shards_are_disjoint_and_cover_the_batch():
    for n in (0, 1, 7, 1000, 1001, 1 << 18):
        for w in (1, 2, 3, 8):
            b = [dp.shard(n, r, w) for r in range(w)]
            assert b[0][0] == 0 and b[-1][1] == n
            assert all(b[r][1] == b[r + 1][0] for r in range(w - 1))
            sizes = [hi - lo for lo, hi in b]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        dp.shard(10, 2, 2)


def test_two_gloo_ranks_equal_one_rank_on_the_whole_batch():
    import oracle as O
    out = _run(2)
    net, params, batches = _problem()
    tr = O.Trainer(net, params, lr=LR)
    want_losses = [tr.step(x, t) for x, t in batches]
    (_, p0, t0, l0), (_, p1, t1, l1) = out
    assert np.array_equal(p0, p1)  # the replicas stay identical
    assert t0 == t1 == 3
    np.testing.assert_allclose(l0, want_losses, rtol=1e-12)
    assert l0 == l1
    # the update is unique where the gradient is clearly away from zero; elsewhere
    # the order of the two halves' sums may pick the other sign of a +-lr move
    moved = np.abs(tr.params - params) > 0
    np.testing.assert_allclose(p0[moved], tr.params[moved], rtol=1e-9, atol=1e-12)
    assert np.all(p0[~moved] == params[~moved])


def test_an_overflow_on_one_rank_skips_the_step_on_every_rank():
    out = _run(2, overflow_rank=1)
    (_, p0, t0, _), (_, p1, t1, _) = out
    assert np.array_equal(p0, p1)
    assert t0 == t1 == 2  # the second of three steps was skipped on both


def test_one_process_needs_no_group():
    net, params, batches = _problem()
    rep = OracleReplica(net, params)
    step = dp.DataParallelStep(rep)
    assert step.world == 1 and step.rank == 0
    import oracle as O
    tr = O.Trainer(net, params, lr=LR)
    x, t = batches[0]
    loss = float(step(torch.from_numpy(x), torch.from_numpy(t))[0])
    assert loss == pytest.approx(tr.step(x, t), rel=1e-12)
    np.testing.assert_allclose(rep.p, tr.params, rtol=1e-12, atol=1e-15)


# ---- image tiles: a frame split by rows over the ranks (dp.render_tiles) ----

def _tile_scene():
    from paper_2207_11620_gb300 import inputs as I
    vol = I.blob_volume(16, seed=2)
    cam = I.perspective_camera(9, 7)  # 7 rows: bands of 4 / 3 and of 3 / 2 / 2
    return vol, cam, I.ramp_lut(), dict(step=0.5 / 16, alpha_exp=0.5, et=0.99)


def _oracle_band(vol, cam, lut, opts):
    import oracle as O
    W = cam["width"]

    def band(row0, rows):
        px = np.arange(row0 * W, (row0 + rows) * W)
        return torch.from_numpy(O.render_pixels(cam, lut, opts, px, vol=vol).reshape(rows, W, 4))
    return band


def _tile_rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    vol, cam, lut, opts = _tile_scene()
    calls = []
    band = _oracle_band(vol, cam, lut, opts)

    def counted(row0, rows):
        calls.append((row0, rows))
        return band(row0, rows)
    img = dp.render_tiles(counted, cam["width"], cam["height"])
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, img.numpy(), calls))


@pytest.mark.parametrize("ws", [2, 3])
def test_gloo_ranks_render_the_frame_by_row_bands(ws):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_tile_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in range(ws)), key=lambda o: o[0])
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    vol, cam, lut, opts = _tile_scene()
    W, H = cam["width"], cam["height"]
    want = _oracle_band(vol, cam, lut, opts)(0, H).numpy()
    assert (want[..., 3] > 0).mean() > 0.2
    for r, img, calls in out:
        assert calls == [(lo, hi - lo) for lo, hi in [dp.shard(H, r, ws)]]  # one band per rank, its own
        assert np.array_equal(img, want)  # every rank holds the whole frame
