"""Parity at the full sizes of configs 4 and 5 (F = 4, T = 2^22 / 2^23, 64-wide
input), in the launch configuration the bench times, on outputs the oracle
computes one by one: network outputs on sampled points, the loss of a full
2^18-point training step on the 1024^3 volume, and ring samples drawn from
64^3 bricks."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2207_11620_gb300 import configs as CF
from paper_2207_11620_gb300 import inputs as I

pytestmark = pytest.mark.gpu

OUT_TOL = 2e-2


@pytest.fixture(scope="module")
def nv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_11620_gb300 import build, nv as nvmod
    build.build()
    return nvmod


def onet(c):
    return O.Net(L=c.L, F=c.F, log2T=c.log2T, Nmin=c.Nmin, b=c.b, dims=c.dims)


def varied(net, c, seed):
    p = I.init_params(net.n_table, net.n_params - net.n_table, seed=seed, dims=c.dims)
    p[: net.n_table] = I.uniform_params(net.n_table, seed=seed + 1, scale=1.0)
    return p


@pytest.mark.parametrize("cfg,prec", [("cfg4", "fp16"), ("cfg5", "bf16")])
def test_full_size_inference_on_sampled_points(nv, cfg, prec):
    c = {"cfg4": CF.CFG4_NET, "cfg5": CF.CFG5_NET}[cfg]
    net = nv.NeuralVolume(prec=prec, **c.kwargs())
    params = varied(net, c, 61)
    net.set_params(params)
    x = I.uniform_points(1 << 16, seed=62)
    x[:3] = [[0, 0, 0], [0.999999, 0.999999, 0.999999], [0.5, 0.25, 0.125]]
    y = net.infer(torch.from_numpy(x).cuda()).cpu().numpy()
    pick = np.random.default_rng(63).choice(x.shape[0], 2048, replace=False)
    pick[:3] = [0, 1, 2]
    want = O.forward(onet(c), params, x[pick])
    assert np.max(np.abs(y[pick] - want)) <= OUT_TOL
    assert want.std() > 0.02


def test_cfg4_training_step_loss_at_full_size(nv):
    """One config-4 step: 2^18 points sampled on the GPU from the 1024^3 volume,
    FP16 MLP; its loss against the oracle's forward over the same points."""
    cfg = CF.CFG4
    c = cfg["net"]
    vt = I.blob_volume_torch(cfg["volume"], cfg["volume_seed"], "cuda")
    net = nv.NeuralVolume(prec="fp16", **c.kwargs())
    params = I.init_params(net.n_table, net.n_params - net.n_table, seed=5, dims=c.dims)
    params[: net.n_table] = I.uniform_params(net.n_table, seed=6, scale=0.5)
    net.set_params(params)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    n = cfg["batch"]
    net.train_step(n=n, vol=vt, seed=41, loss_out=loss)
    x = O.sample_points(41, 0, 0, n)
    # the targets: trilinear values of the GPU-generated volume at the oracle's points
    vol = vt.cpu().numpy()
    del vt
    torch.cuda.empty_cache()
    t = O.trilinear(vol, x).astype(np.float32)
    y = O.forward(onet(c), params, x)
    lo = O.loss_l2(y, t)
    assert abs(loss.item() - lo) <= OUT_TOL * lo, (loss.item(), lo)
    step, _ = net.step_info()
    assert step == 1


def test_cfg5_ring_of_64_cubed_bricks_matches_oracle(nv):
    vol = I.blob_volume(256, seed=6)
    host = torch.from_numpy(I.host_bricks(vol, 64)).pin_memory()
    ring = nv.BrickRing(host, vol.shape, brick=64, ring_slots=24, seed=3)
    n = 50000
    for step, refresh in ((0, 0), (1, 16)):
        if refresh:
            ring.refresh(refresh, seed=7)
        slots = ring.slots()
        xyz, t = ring.sample(n, seed=11, step=step)
        ox, ot = O.brick_sample(vol, 64, np.array(slots, np.int32), 11, step, n)
        np.testing.assert_array_equal(xyz.cpu().numpy(), ox)
        got = t.cpu().numpy().astype(np.float64)
        # trilinear of voxels >= 0: the error magnitude is the value itself
        assert np.all(np.abs(got - ot) <= 1e-5 * np.abs(ot))
    ring.close()
