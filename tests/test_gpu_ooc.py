"""GPU parity of the out-of-core sampling ring (A-17, Sec. 4.1) against the oracle:
the sampled points are bit-exact and the targets within FP32 rounding of the
volume's trilinear values, for the ring as created and after a refresh."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2207_11620_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_11620_gb300 import build, nv as nvmod
    build.build()
    return nvmod


def test_device_brick_layout_matches_host():
    vol = I.blob_volume((32, 48, 64), seed=2)
    want = I.host_bricks(vol, 16)
    got = I.host_bricks_from_device(torch.from_numpy(vol).cuda(), 16)
    np.testing.assert_array_equal(got.numpy(), want)


def test_ring_samples_match_oracle(nv):
    vol = I.blob_volume((32, 48, 64), seed=7)
    host = torch.from_numpy(I.host_bricks(vol, 16)).pin_memory()
    ring = nv.BrickRing(host, vol.shape, brick=16, ring_slots=6, seed=5)
    n = 20000 + 3
    for step, refresh in ((0, 0), (1, 3), (2, 6)):
        if refresh:
            ring.refresh(refresh, seed=100 + step)
        slots = ring.slots()
        xyz, t = ring.sample(n, seed=9, step=step)
        ox, ot = O.brick_sample(vol, 16, np.array(slots, np.int32), 9, step, n)
        np.testing.assert_array_equal(xyz.cpu().numpy(), ox)
        got = t.cpu().numpy().astype(np.float64)
        # trilinear of voxels >= 0: the error magnitude is the value itself
        assert np.all(np.abs(got - ot) <= 1e-5 * np.abs(ot))
    b, ms = ring.stats()
    assert b == (3 + 6) * 18 ** 3 * 4
    ring.close()


def test_ring_training_reduces_loss(nv):
    from paper_2207_11620_gb300 import configs as CF
    vol = I.blob_volume(64, seed=3)
    host = torch.from_numpy(I.host_bricks(vol, 16)).pin_memory()
    ring = nv.BrickRing(host, vol.shape, brick=16, ring_slots=16, seed=1)
    c = CF.CFG2_NET
    net = nv.NeuralVolume(prec="bf16", **c.kwargs())
    net.set_params(I.init_params(net.n_table, net.n_params - net.n_table, seed=4, dims=c.dims))
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    xyz = torch.empty((1 << 14, 3), dtype=torch.float32, device="cuda")
    tgt = torch.empty(1 << 14, dtype=torch.float32, device="cuda")
    hist = []
    for s in range(80):
        ring.sample(1 << 14, seed=3, step=s, xyz=xyz, target=tgt)
        ring.refresh(4, seed=s)
        net.train_step(xyz, tgt, loss_out=loss)
        hist.append(loss.item())
    assert hist[-1] < 0.3 * hist[0]
    ring.close()


def test_ring_rejects_bad_arguments(nv):
    vol = I.blob_volume(16, seed=1)
    host = torch.from_numpy(I.host_bricks(vol, 8)).pin_memory()
    with pytest.raises(nv.NvError, match="ring_slots"):
        nv.BrickRing(host, vol.shape, brick=8, ring_slots=9)
    with pytest.raises(nv.NvError, match="multiple"):
        nv.BrickRing(host, vol.shape, brick=6, ring_slots=2)
    with pytest.raises(ValueError):
        nv.BrickRing(torch.from_numpy(I.host_bricks(vol, 8)), vol.shape, brick=8, ring_slots=2)
