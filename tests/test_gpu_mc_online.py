"""GPU parity of online macrocell construction (Sec. 5.3): value ranges grown
from training samples and mu_max from those ranges, against the oracle.
Ranges are min / max of FP32 sample values, so they match bit for bit when
both sides see the same values."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2207_11620_gb300 import configs as CF
from paper_2207_11620_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_11620_gb300 import build, nv as nvmod
    build.build()
    return nvmod


def _samples(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.random((n, 3), dtype=np.float32)
    e = np.float32(1.0) - np.float32(2 ** -24)
    x[:6] = [[0, 0, 0], [e, e, e], [1, 1, 1], [0.125, 0.125, 0.125], [0.5, 0.25, e], [0, e, 0.5]]
    v = rng.uniform(-0.25, 1.25, n).astype(np.float32)  # outside [0, 1] too: mu clamps
    return x, v


@pytest.mark.parametrize("shape,cell", [((40, 33, 50), 8), ((64, 64, 64), 16), ((17, 9, 5), 4)])
def test_update_and_mu_bit_exact(nv, shape, cell):
    lut = I.ramp_lut(alpha_floor=0.3)
    mm = nv.online_macrocells(shape, cell)
    want = O.mc_online_empty(shape, cell)
    for b in range(3):  # several batches accumulate
        x, v = _samples(20000 + 7 * b, seed=b)
        nv.macrocells_update(mm, torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda(), shape, cell)
        O.mc_online_update(want, x, v, shape, cell)
    np.testing.assert_array_equal(mm.cpu().numpy(), want)
    mu = nv.macrocells_mu(mm, shape, cell, torch.from_numpy(lut).cuda())
    np.testing.assert_array_equal(mu.cpu().numpy(), O.mc_mu(want, lut))


def test_empty_cells_are_skipped(nv):
    shape, cell = (32, 32, 32), 8
    mm = nv.online_macrocells(shape, cell)
    x = np.array([[0.1, 0.1, 0.1]], np.float32)
    nv.macrocells_update(mm, torch.from_numpy(x).cuda(), torch.tensor([0.7], device="cuda"), shape, cell)
    mu = nv.macrocells_mu(mm, shape, cell, torch.from_numpy(I.ramp_lut()).cuda()).cpu().numpy()
    assert mu[0, 0, 0] == pytest.approx(np.float32(179 / 255), abs=1e-6)  # ceil(255 * 0.7) = 179
    assert np.count_nonzero(mu) == 1


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_train_step_widens_registered_ranges(nv, prec):
    """Host batches: the ranges after three steps are exactly the oracle's over
    the same points and targets; sampled batches: within the rounding of the
    FP32 trilinear target."""
    c = CF.CFG2_NET
    vol = I.blob_volume(48, seed=2)
    shape, cell = vol.shape, 16
    net = nv.NeuralVolume(prec=prec, **c.kwargs())
    net.set_params(I.init_params(net.n_table, net.n_params - net.n_table, seed=1, dims=c.dims))
    mm = nv.online_macrocells(shape, cell)
    net.set_online_macrocells(mm, shape, cell)
    want = O.mc_online_empty(shape, cell)
    for s in range(3):
        x = O.sample_points(40, s, 0, 4096)
        t = O.trilinear(vol, x).astype(np.float32)
        net.train_step(torch.from_numpy(x), torch.from_numpy(t))
        O.mc_online_update(want, x, t, shape, cell)
    np.testing.assert_array_equal(mm.cpu().numpy(), want)
    # sampled batches (the context's sampler counter starts at 0)
    mm2 = nv.online_macrocells(shape, cell)
    net.set_online_macrocells(mm2, shape, cell)
    vt = torch.from_numpy(vol).cuda()
    want2 = O.mc_online_empty(shape, cell)
    for s in range(2):
        net.train_step(n=8192, vol=vt, seed=77)
        x = O.sample_points(77, s, 0, 8192)
        O.mc_online_update(want2, x, O.trilinear(vol, x).astype(np.float32), shape, cell)
    got = mm2.cpu().numpy()
    np.testing.assert_array_equal(np.isfinite(got), np.isfinite(want2))
    f = np.isfinite(want2)
    assert np.max(np.abs(got[f] - want2[f])) <= 1e-6
    net.set_online_macrocells(None)
    net.train_step(n=1024, vol=vt, seed=78)
    np.testing.assert_array_equal(mm2.cpu().numpy(), got)  # no longer widened


def test_online_macrocells_render_close_to_precomputed(nv):
    """Sec. 5.3: rendering with ranges grown during training loses little
    against ranges precomputed from the voxels."""
    c = CF.CFG2_NET
    vol = I.blob_volume(64, seed=3)
    vt = torch.from_numpy(vol).cuda()
    shape, cell = vol.shape, 8
    net = nv.NeuralVolume(prec="fp16", **c.kwargs())
    net.set_params(I.init_params(net.n_table, net.n_params - net.n_table, seed=4, dims=c.dims))
    mm = nv.online_macrocells(shape, cell)
    net.set_online_macrocells(mm, shape, cell)
    for s in range(300):
        net.train_step(n=1 << 14, vol=vt, seed=5)
    lut = torch.from_numpy(I.ramp_lut(alpha_floor=0.1)).cuda()
    mu_on = nv.macrocells_mu(mm, shape, cell, lut)
    _, mu_pre = nv.macrocells_build(vt, cell, lut)
    assert torch.all(mu_on <= mu_pre)
    cam = I.perspective_camera(128, 96)
    opts = dict(step=0.5 / 64, alpha_exp=0.5, et=0.99, K=8)
    r = nv.Renderer(128 * 96, K=8)
    raw = r.render(cam, lut, opts, raw=vt, mc=(mu_pre, cell, shape)).clone()
    img_pre = r.render(cam, lut, opts, net=net, mc=(mu_pre, cell, shape)).clone()
    img_on = r.render(cam, lut, opts, net=net, mc=(mu_on, cell, shape)).clone()

    def psnr(a, b):
        return 10 * np.log10(1.0 / nv.image_mse(a, b).item())
    p_pre, p_on = psnr(img_pre, raw), psnr(img_on, raw)
    assert p_pre > 30
    assert p_on > p_pre - 1.0, (p_on, p_pre)
