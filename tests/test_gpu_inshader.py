"""GPU parity of the in-shader ray march (Sec. 5.1, App. A): the megakernel
takes the samples of the sample-streaming march, evaluates the same network
arithmetic and composites the same way, so its image equals nv_render's; both
are checked against the oracle's ray march."""
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


def onet(c):
    return O.Net(L=c.L, F=c.F, log2T=c.log2T, Nmin=c.Nmin, b=c.b, dims=c.dims)


def varied_params(net, c, seed):
    p = I.init_params(net.n_table, net.n_params - net.n_table, seed=seed, dims=c.dims)
    p[: net.n_table] = I.uniform_params(net.n_table, seed=seed + 1, scale=1.0)
    return p


SMALL_F4 = CF.NetCfg(16, 4, 14, 16, 1.38, (64, 64, 64, 1))


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("shape", ["cfg1", "cfg2", "f4d64"])
def test_inshader_equals_streaming_ortho(nv, prec, shape):
    c = {"cfg1": CF.CFG1_NET, "cfg2": CF.CFG2_NET, "f4d64": SMALL_F4}[shape]
    net = nv.NeuralVolume(prec=prec, **c.kwargs())
    net.set_params(varied_params(net, c, 46))
    cam = I.ortho_camera_z(70, 37)  # 2590 rays: 21 CTAs, the last one ragged
    lut = torch.from_numpy(I.ramp_lut()).cuda()
    opts = dict(step=1 / 128, alpha_exp=1.0, et=0.99, K=8)
    ss = nv.Renderer(70 * 37, K=8).render(cam, lut, opts, net=net)
    sam = torch.zeros(1, dtype=torch.int64, device="cuda")
    is_ = nv.render_inshader(net, cam, lut, opts, samples=sam)
    torch.cuda.synchronize()
    d = (is_ - ss).abs().max().item()
    assert d <= 1e-6, d
    assert 0 < sam.item() <= 70 * 37 * 128


def test_streaming_over_several_inference_chunks_equals_inshader(nv):
    """A 1280 x 1024 orthographic frame over the unit square: 1.3 M rays,
    10.5 M samples in the first streaming iteration at K = 8, which the
    tensor-core path takes in two inference chunks (2^23 points each at most);
    the in-shader kernel evaluates the same samples without chunks."""
    c = CF.CFG2_NET
    net = nv.NeuralVolume(prec="fp16", **c.kwargs())
    net.set_params(varied_params(net, c, 52))
    W, H = 1280, 1024
    cam = I.ortho_camera_z(W, H)
    lut = torch.from_numpy(I.ramp_lut()).cuda()
    opts = dict(step=1 / 128, alpha_exp=1.0, et=0.99, K=8)
    r = nv.Renderer(W * H, K=8)
    ss = r.render(cam, lut, opts, net=net)
    it, ns = r.stats()
    is_ = nv.render_inshader(net, cam, lut, opts)
    torch.cuda.synchronize()
    assert ns >= W * H * 8 > (1 << 23)  # the first iteration alone: 8 samples of every ray
    d = (is_ - ss).abs().max().item()
    assert d <= 1e-6, d


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_inshader_perspective_macrocells_matches_streaming_and_oracle(nv, prec):
    c = CF.CFG2_NET
    net = nv.NeuralVolume(prec=prec, **c.kwargs())
    params = I.init_params(net.n_table, net.n_params - net.n_table, seed=5, dims=c.dims)
    vol = I.blob_volume((40, 48, 56), seed=9)
    vt = torch.from_numpy(vol).cuda()
    net.set_params(params)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    for s in range(150):  # a network that resembles the volume, so macrocells matter
        net.train_step(n=1 << 14, vol=vt, seed=3, loss_out=loss)
    lut_np = I.ramp_lut(alpha_floor=0.1)
    lut = torch.from_numpy(lut_np).cuda()
    mm, mu = nv.macrocells_build(vt, 8, lut)
    mc = (mu, 8, vol.shape)
    cam = I.perspective_camera(96, 64)
    opts = dict(step=0.5 / 56, alpha_exp=0.5, et=0.99, K=8, mc_cell=8)
    ss = nv.Renderer(96 * 64, K=8).render(cam, lut, opts, net=net, mc=mc)
    is_ = nv.render_inshader(net, cam, lut, opts, mc=mc)
    torch.cuda.synchronize()
    d = (is_ - ss).abs().max().item()
    assert d <= 1e-6, d
    # against the oracle's march on the trained parameters, sampled pixels
    got_params = net.get_params().cpu().numpy()
    pix = np.random.default_rng(1).choice(96 * 64, 300, replace=False)
    mu_o = O.macrocells(vol, 8, lut_np)[1]
    np.testing.assert_array_equal(mu_o, mu.cpu().numpy())
    want = O.render_pixels(cam, lut_np, opts, pix, net=onet(c), params=got_params, vol=vol, mumax=mu_o)
    got = is_.cpu().numpy().reshape(-1, 4)[pix]
    assert np.max(np.abs(got - want)) <= 5e-2


def test_inshader_rejects_fp32_network(nv):
    c = CF.CFG1_NET
    net = nv.NeuralVolume(prec="fp32", **c.kwargs())
    net.set_params(I.uniform_params(net.n_params, seed=1))
    lut = torch.from_numpy(I.ramp_lut()).cuda()
    with pytest.raises(nv.NvError, match="FP16 or BF16"):
        nv.render_inshader(net, I.ortho_camera_z(8, 8), lut, dict(step=1 / 128))
