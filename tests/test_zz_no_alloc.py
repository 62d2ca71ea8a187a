"""nv_render_raw_noalloc: the raw-volume ray march for callers that cannot
allocate device memory (real-time loops with a fixed memory budget, where an
allocation may synchronise the device mid-frame; plugins whose host
application owns every allocation), with its scratch in a static device array.
It runs the same kernels as nv_render (the renderer-object entry point) and
every pixel is composited on its own, so its images must equal nv_render's bit
for bit, on two calls in a row with different image sizes, K and macrocell use:
leftovers of the first call in the shared scratch cannot leak into the second.
Named to run after every other test file."""
import ctypes as C

import pytest
import torch

from paper_2207_11620_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_11620_gb300 import build, nv as nvmod
    build.build()
    return nvmod


def render_noalloc(nvmod, vol, cam, lut, opts, mc=None):
    out = torch.full((cam["height"], cam["width"], 4), float("nan"), dtype=torch.float32, device="cuda")
    v = nvmod.volume(vol)
    c = nvmod.camera(cam)
    o = nvmod.RenderOpts(float(opts["step"]), float(opts["alpha_exp"]), float(opts["et"]), int(opts["K"]))
    mp = None
    if mc is not None:
        mu, cell = mc
        nz, ny, nx = vol.shape
        m = nvmod.Macrocells(mu.data_ptr(), int(cell), int(nx), int(ny), int(nz))
        mp = C.byref(m)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = nvmod.lib().nv_render_raw_noalloc(C.byref(v), C.byref(c), C.c_void_p(lut.data_ptr()), mp, C.byref(o),
                                           C.c_void_p(out.data_ptr()), stream)
    assert st == 0, nvmod.lib().nv_last_error().decode()
    torch.cuda.synchronize()
    return out


def test_noalloc_render_matches_renderer_on_two_calls(nv):
    vol = torch.from_numpy(I.blob_volume(40, seed=4)).cuda()
    lut = torch.from_numpy(I.ramp_lut(alpha_floor=0.1)).cuda()
    _, mu = nv.macrocells_build(vol, 8, lut)
    cases = [
        (I.perspective_camera(160, 120), dict(step=0.5 / 40, alpha_exp=0.5, et=0.99, K=8), (mu, 8)),
        (I.ortho_camera_z(200, 150), dict(step=1.0 / 64, alpha_exp=1.0, et=0.95, K=4), None),
    ]
    for cam, opts, mc in cases:
        got = render_noalloc(nv, vol, cam, lut, opts, mc)
        r = nv.Renderer(cam["width"] * cam["height"], K=opts["K"])
        want = r.render(cam, lut, opts, raw=vol, mc=(mc[0], mc[1], vol.shape) if mc else None)
        torch.cuda.synchronize()
        assert torch.isfinite(got).all().item()
        assert torch.equal(got, want)
        assert (want[..., 3] > 0).float().mean().item() > 0.2
        r.close()


def test_noalloc_rejects_images_over_the_static_maximum(nv):
    vol = torch.from_numpy(I.blob_volume(16, seed=1)).cuda()
    lut = torch.from_numpy(I.ramp_lut()).cuda()
    cam = I.perspective_camera(257, 256)
    with pytest.raises(AssertionError, match="exceeds the static maximum"):
        render_noalloc(nv, vol, cam, lut, dict(step=1 / 32, alpha_exp=1.0, et=0.99, K=8))


@pytest.mark.parametrize("field", ["step_max", "shade"])
def test_noalloc_refuses_adaptive_step_and_shadows(nv, field):
    vol = torch.from_numpy(I.blob_volume(16, seed=1)).cuda()
    lut = torch.from_numpy(I.ramp_lut()).cuda()
    cam = nv.camera(I.perspective_camera(32, 32))
    o = nv.RenderOpts(1.0 / 32, 1.0, 0.99, 8)
    setattr(o, field, 16.0 / 16 if field == "step_max" else 1)
    out = torch.zeros((32, 32, 4), dtype=torch.float32, device="cuda")
    v = nv.volume(vol)
    st = nv.lib().nv_render_raw_noalloc(C.byref(v), C.byref(cam), C.c_void_p(lut.data_ptr()), None, C.byref(o),
                                        C.c_void_p(out.data_ptr()), C.c_void_p(0))
    assert st == 6  # NV_ERR_UNSUPPORTED, before anything is enqueued
    assert "fixed step only" in nv.lib().nv_last_error().decode()
    assert torch.count_nonzero(out).item() == 0
