"""Image-tile split of the ray march (nv_render_rows, dp.render_tiles): each
pixel's ray is marched and composited on its own (Sec. 5.2.1), so a band of
rows rendered alone must equal those rows of the whole frame bit for bit --
on the raw volume and through the FP16 tensor-core network, with macrocell
skipping, the adaptive step and single-shot shadows, and for bands that do
not divide the image evenly.  The whole frame itself is checked against the
oracle by the parity tests; here the band of rows at an offset is also checked
against the oracle directly, so the row offset of the rays is pinned by
something other than the renderer."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2207_11620_gb300 import configs as CF, dp, inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_11620_gb300 import build, nv as nvmod
    build.build()
    return nvmod


@pytest.fixture(scope="module")
def scene(nv):
    vol = I.blob_volume((40, 48, 56), seed=4)
    vt = torch.from_numpy(vol).cuda()
    lut = I.ramp_lut_soft(0.1)
    lt = torch.from_numpy(lut).cuda()
    _, mu = nv.macrocells_build(vt, 8, lt)
    return vol, vt, lut, lt, mu


def _bands(height, parts):
    return [dp.shard(height, r, parts) for r in range(parts)]


def _net(nv):
    c = CF.CFG2_NET
    net = nv.NeuralVolume(prec="fp16", **c.kwargs())
    params = I.init_params(net.n_table, net.n_params - net.n_table, seed=7, dims=c.dims)
    params[: net.n_table] = I.uniform_params(net.n_table, seed=8, scale=0.5)
    net.set_params(params)
    return net


@pytest.mark.parametrize("mode", ["fixed", "adaptive", "shadows"])
@pytest.mark.parametrize("source", ["raw", "fp16"])
def test_row_bands_equal_the_whole_frame(nv, scene, mode, source):
    vol, vt, lut, lt, mu = scene
    W, H = 72, 55  # 55 rows: bands of 19 / 18 / 18 and of 14 / 14 / 14 / 13
    s1 = 0.5 / 56
    opts = dict(step=s1, alpha_exp=0.5, et=0.99, K=8)
    if mode == "adaptive":
        opts["step_max"] = 16 * s1
    if mode == "shadows":
        opts.update(shade=1, light=(0.48, 0.6, -0.64), ambient=0.25)
    cam = I.perspective_camera(W, H)
    net = _net(nv) if source == "fp16" else None
    raw = vt if net is None else None
    mc = (mu, 8, vol.shape)
    r = nv.Renderer(W * H, K=8)
    whole = r.render(cam, lt, opts, net=net, raw=raw, mc=mc).clone()
    assert (whole[..., 3] > 0).float().mean().item() > 0.2
    for parts in (1, 3, 4):
        got = torch.cat([r.render(cam, lt, opts, net=net, raw=raw, mc=mc, rows=(a, b - a)).clone()
                         for a, b in _bands(H, parts)], dim=0)
        assert torch.equal(got, whole), (parts, (got - whole).abs().max().item())
    r.close()


def test_a_band_at_an_offset_matches_the_oracle(nv, scene):
    vol, vt, lut, lt, mu = scene
    W, H = 64, 48
    opts = dict(step=0.5 / 56, alpha_exp=0.5, et=0.99, K=8, mc_cell=8)
    cam = I.perspective_camera(W, H)
    r = nv.Renderer(W * 20, K=8)  # room for the band only
    band = r.render(cam, lt, opts, raw=vt, mc=(mu, 8, vol.shape), rows=(17, 20)).cpu().numpy().reshape(-1, 4)
    want, mag = O.render_pixels(cam, lut, opts, np.arange(17 * W, 37 * W), vol=vol, mumax=mu.cpu().numpy(),
                                with_mag=True)
    # FP32 march against the FP64 oracle: |g - o| <= 1e-5 M per channel, except
    # pixels whose opacity is within rounding of the early-termination threshold
    # (one sample more or less on one side moves them by at most 1 - et), which
    # must be rare
    got = band.astype(np.float64)
    err = np.abs(got - want)
    bad = np.any(err > 1e-5 * mag, axis=1)
    term = np.maximum(got[:, 3], want[:, 3]) >= opts["et"] - 1e-4
    assert not np.any(bad & ~term)
    assert (bad & term).sum() <= max(2, 0.01 * len(want))
    assert np.all(err[bad] <= 1.0 - opts["et"] + 1e-5)
    assert (band[:, 3] > 0).mean() > 0.2
    r.close()


def test_render_tiles_without_a_group_renders_the_frame(nv, scene):
    vol, vt, lut, lt, mu = scene
    W, H = 40, 30
    opts = dict(step=0.5 / 56, alpha_exp=0.5, et=0.99, K=8)
    cam = I.perspective_camera(W, H)
    r = nv.Renderer(W * H, K=8)
    whole = r.render(cam, lt, opts, raw=vt).clone()
    img = dp.render_tiles(lambda a, n: r.render(cam, lt, opts, raw=vt, rows=(a, n)), W, H)
    assert torch.equal(img, whole)
    r.close()


@pytest.mark.parametrize("rows", [(-1, 4), (0, 0), (28, 3), (0, 31)])
def test_bands_outside_the_image_are_refused(nv, scene, rows):
    vol, vt, lut, lt, mu = scene
    cam = I.perspective_camera(40, 30)
    r = nv.Renderer(40 * 30, K=8)
    out = torch.zeros((max(rows[1], 1), 40, 4), device="cuda")
    with pytest.raises(RuntimeError, match="not inside the image"):
        r.render(cam, lt, dict(step=0.01, alpha_exp=1.0, et=0.99, K=8), raw=vt, rows=rows, out=out)
    r.close()


def test_a_band_larger_than_the_renderer_is_refused(nv, scene):
    vol, vt, lut, lt, mu = scene
    cam = I.perspective_camera(40, 30)
    r = nv.Renderer(40 * 10, K=8)
    r.render(cam, lt, dict(step=0.01, alpha_exp=1.0, et=0.99, K=8), raw=vt, rows=(20, 10))
    with pytest.raises(RuntimeError, match="exceed the renderer"):
        r.render(cam, lt, dict(step=0.01, alpha_exp=1.0, et=0.99, K=8), raw=vt, rows=(5, 11))
    r.close()
