"""GPU parity of the adaptive-step ray march (Sec. 5.3, Eq. 3) against the
oracle: the segment boundaries and sample positions are the same FP32
operations on both sides, values follow the FP32 tolerance.  The transfer
function is transparent below 0.1 and rises linearly from there
(ramp_lut_soft): a LUT that jumps at the floor multiplies the FP32 rounding of
a sample value by its slope (26 at a jump of 0.1 over one entry), which the
FP32 tolerance of the path does not cover."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2207_11620_gb300 import configs as CF
from paper_2207_11620_gb300 import inputs as I
from tests.test_gpu_parity import _compare_images

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_11620_gb300 import build, nv as nvmod
    build.build()
    return nvmod


def onet(c):
    return O.Net(L=c.L, F=c.F, log2T=c.log2T, Nmin=c.Nmin, b=c.b, dims=c.dims)


@pytest.mark.parametrize("cell,smax", [(8, 16.0), (4, 64.0), (16, 1.0)])
@pytest.mark.parametrize("K", [1, 8])
def test_adaptive_raw_volume_matches_oracle(nv, cell, smax, K):
    vol = I.blob_volume((40, 48, 56), seed=4)
    vt = torch.from_numpy(vol).cuda()
    lut = I.ramp_lut_soft(0.1)
    lt = torch.from_numpy(lut).cuda()
    _, mu = nv.macrocells_build(vt, cell, lt)
    if cell <= 8:
        assert (mu == 0).float().mean().item() > 0.1  # transparent cells to cross
    s1 = 0.5 / 56
    opts = dict(step=s1, step_max=s1 * smax, alpha_exp=0.5, et=0.99, K=K, mc_cell=cell)
    cam = I.perspective_camera(80, 60)
    r = nv.Renderer(80 * 60, K=K)
    img = r.render(cam, lt, opts, raw=vt, mc=(mu, cell, vol.shape)).cpu().numpy()
    want = O.render_pixels(cam, lut, opts, np.arange(80 * 60), vol=vol, mumax=mu.cpu().numpy(), with_mag=True)
    _compare_images(img, want)
    assert want[0][:, 3].max() > 0.5


def test_adaptive_network_fp32_matches_oracle(nv):
    c = CF.CFG2_NET
    net = nv.NeuralVolume(prec="fp32", **c.kwargs())
    params = I.init_params(net.n_table, net.n_params - net.n_table, seed=7, dims=c.dims)
    params[: net.n_table] = I.uniform_params(net.n_table, seed=8, scale=0.5)
    net.set_params(params)
    vol = I.blob_volume(32, seed=5)
    lut = I.ramp_lut_soft(0.1)
    lt = torch.from_numpy(lut).cuda()
    _, mu = nv.macrocells_build(torch.from_numpy(vol).cuda(), 8, lt)
    opts = dict(step=0.5 / 32, step_max=8 / 32, alpha_exp=0.5, et=0.99, K=8, mc_cell=8)
    cam = I.perspective_camera(48, 40)
    img = nv.Renderer(48 * 40, K=8).render(cam, lt, opts, net=net, mc=(mu, 8, vol.shape)).cpu().numpy()
    pix = np.random.default_rng(2).choice(48 * 40, 400, replace=False)
    want = O.render_pixels(cam, lut, opts, pix, net=onet(c), params=params, vol=vol, mumax=mu.cpu().numpy(),
                           with_mag=True)
    _compare_images(img.reshape(-1, 4)[pix], want)


def test_adaptive_constant_medium_closed_form(nv):
    n = 32
    vol = np.full((n, n, n), np.float32(100 / 255), np.float32)
    lut = I.ramp_lut()
    lt = torch.from_numpy(lut).cuda()
    vt = torch.from_numpy(vol).cuda()
    _, mu = nv.macrocells_build(vt, 8, lt)
    s1 = 0.5 / n
    opts = dict(step=s1, step_max=32 * s1, alpha_exp=0.5, et=2.0, K=8)
    cam = I.perspective_camera(16, 12)
    img = nv.Renderer(16 * 12, K=8).render(cam, lt, opts, raw=vt, mc=(mu, 8, vol.shape)).cpu().numpy()
    a = float(lut[100, 3])
    for p in range(16 * 12):
        hit, o, d, t01 = O.pixel_ray(cam, p % 16, p // 16)
        if not hit:
            assert np.all(img.reshape(-1, 4)[p] == 0)
            continue
        A = 1.0 - (1.0 - a) ** ((float(t01[1]) - float(t01[0])) * n)
        assert img.reshape(-1, 4)[p, 3] == pytest.approx(A, abs=1e-4)


def test_adaptive_takes_fewer_samples(nv):
    vol = I.blob_volume(48, seed=4)
    vt = torch.from_numpy(vol).cuda()
    lt = torch.from_numpy(I.ramp_lut(alpha_floor=0.1)).cuda()
    _, mu = nv.macrocells_build(vt, 8, lt)
    cam = I.perspective_camera(64, 48)
    r = nv.Renderer(64 * 48, K=8)
    base = dict(step=0.5 / 48, alpha_exp=0.5, et=0.99, K=8)
    r.render(cam, lt, base, raw=vt, mc=(mu, 8, vol.shape))
    n_fixed = r.stats()[1]
    r.render(cam, lt, dict(base, step_max=32 / 48), raw=vt, mc=(mu, 8, vol.shape))
    n_adapt = r.stats()[1]
    assert 0 < n_adapt < 0.8 * n_fixed, (n_adapt, n_fixed)


def test_adaptive_needs_macrocells(nv):
    vt = torch.from_numpy(I.blob_volume(16, seed=1)).cuda()
    lt = torch.from_numpy(I.ramp_lut()).cuda()
    r = nv.Renderer(64, K=8)
    with pytest.raises(nv.NvError, match="macrocells"):
        r.render(I.ortho_camera_z(8, 8), lt, dict(step=1 / 64, step_max=1 / 8), raw=vt)
