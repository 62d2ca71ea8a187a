"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: hash indices and macrocell bounds bit-exact; the FP32 path within
1e-5 relative error per element, relative to the element's error magnitude
M >= |o|, the Sum |terms| the oracle propagates with it (oracle/oracle.c,
"error magnitudes"; pinned by tests/test_oracle_magnitudes.py):
|g - o| <= 1e-5 M.  Where nothing cancels M = |o| and this is the plain
relative bound; where a sum cancels, FP32 rounding scales with its terms, and
M says by how much, element by element.  Gradient checks take points whose
ReLU pre-activations are clear of zero by more than that bound (|z| > 1e-5
M(z)): elsewhere a unit's mask, and with it the gradient, is not decided by
the arithmetic.  The scalar reductions (image and volume MSE) are checked
relative to their value.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2207_11620_gb300 import configs as CF
from paper_2207_11620_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def mag_err(g, o, m):
    """max |g - o| / M over the elements; an element with M = 0 must be exact."""
    g = np.asarray(g, np.float64).ravel()
    o = np.asarray(o, np.float64).ravel()
    m = np.asarray(m, np.float64).ravel()
    if o.size == 0:
        return 0.0
    d = np.abs(g - o)
    assert np.all(d[m == 0] == 0), "an element with zero magnitude differs"
    nz = m > 0
    return float(np.max(d[nz] / m[nz])) if nz.any() else 0.0


def kink_free(net, params, x, tol=FP32_TOL):
    """Points none of whose hidden pre-activations lies within tol M(z) of zero."""
    return O.forward_mag(net, params, x)[2] > tol


@pytest.fixture(scope="module")
def nv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_11620_gb300 import build, nv as nvmod
    build.build()
    return nvmod


def make_net(nvmod, cfg, prec="fp32"):
    return nvmod.NeuralVolume(prec=prec, **cfg.kwargs())


def onet(cfg):
    return O.Net(L=cfg.L, F=cfg.F, log2T=cfg.log2T, Nmin=cfg.Nmin, b=cfg.b, dims=cfg.dims)


def edge_points():
    e = np.float32(1.0) - np.float32(2 ** -24)
    return np.array([[0, 0, 0], [e, e, e], [1, 1, 1], [0.5, 0.25, 0.125], [e, 0, 0.5]], np.float32)


# -------------------------------------------------------------- encoding ----

@pytest.mark.parametrize("cfg", [CF.CFG1_NET, CF.CFG2_NET])
def test_hash_indices_bit_exact(nv, cfg):
    net = make_net(nv, cfg)
    x = np.concatenate([I.uniform_points((1 << 14) + 37, seed=5), edge_points()])
    got = net.hash_indices(torch.from_numpy(x).cuda()).cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(got, O.hash_indices(onet(cfg), x))
    assert net.res == list(O.level_res(cfg.L, cfg.Nmin, cfg.b))


@pytest.mark.parametrize("cfg", [CF.CFG1_NET, CF.CFG2_NET])
def test_encode_matches_oracle(nv, cfg):
    net = make_net(nv, cfg)
    params = I.uniform_params(net.n_params, seed=1)
    net.set_params(params)
    x = np.concatenate([I.uniform_points(20000 + 13, seed=6), edge_points()])
    got = net.encode(torch.from_numpy(x).cuda()).cpu().numpy()
    want = O.encode(onet(cfg), params, x)
    assert mag_err(got, want, O.encode_mag(onet(cfg), params, x)) <= FP32_TOL


# --------------------------------------------------------------- network ----

def test_infer_cfg1_full_size(nv):
    cfg = CF.CFG1
    net = make_net(nv, cfg["net"])
    params = I.uniform_params(net.n_params, seed=cfg["param_seed"])
    net.set_params(params)
    x = I.uniform_points(cfg["n_points"], seed=cfg["point_seed"])
    got = net.infer(torch.from_numpy(x).cuda()).cpu().numpy()
    want, wmag, _ = O.forward_mag(onet(cfg["net"]), params, x)
    assert mag_err(got, want, wmag) <= FP32_TOL


def test_infer_varied_outputs(nv):
    cfg = CF.CFG1_NET
    net = make_net(nv, cfg)
    params = I.uniform_params(net.n_params, seed=31, scale=1.0)
    net.set_params(params)
    x = I.uniform_points(50000, seed=32)
    got = net.infer(torch.from_numpy(x).cuda()).cpu().numpy()
    want, wmag, _ = O.forward_mag(onet(cfg), params, x)
    assert np.std(want) > 0.05
    assert mag_err(got, want, wmag) <= FP32_TOL


@pytest.mark.parametrize("n", [0, 1, 127, 129, 1000])
def test_infer_ragged_and_empty(nv, n):
    cfg = CF.CFG2_NET
    net = make_net(nv, cfg)
    params = I.uniform_params(net.n_params, seed=3)
    net.set_params(params)
    x = I.uniform_points(n, seed=n + 1)
    got = net.infer(torch.from_numpy(x).cuda().reshape(n, 3)).cpu().numpy()
    if n:
        want, wmag, _ = O.forward_mag(onet(cfg), params, x)
        assert mag_err(got, want, wmag) <= FP32_TOL


def test_backward_matches_oracle(nv):
    cfg = CF.CFG2_NET
    net = make_net(nv, cfg)
    params = I.uniform_params(net.n_params, seed=4)
    net.set_params(params)
    x = I.uniform_points(3000, seed=7)
    x = x[kink_free(onet(cfg), params, x)]
    n = x.shape[0]
    assert n > 2800
    dy = np.random.default_rng(8).normal(size=n).astype(np.float32)
    g = torch.zeros(net.n_params, dtype=torch.float32, device="cuda")
    net.backward(torch.from_numpy(x).cuda(), torch.from_numpy(dy).cuda(), g)
    want = O.backward(onet(cfg), params, x, dy.astype(np.float64))
    gmag = O.backward_mag(onet(cfg), params, x, np.abs(dy.astype(np.float64)))
    got = g.cpu().numpy()
    nt = net.n_table
    assert mag_err(got[nt:], want[nt:], gmag[nt:]) <= FP32_TOL
    assert mag_err(got[:nt], want[:nt], gmag[:nt]) <= FP32_TOL
    # untouched table entries stay exactly zero
    assert np.all(got[:nt][want[:nt] == 0] == 0)


def test_autograd_function_l1_loss(nv):
    # a loss the library does not implement itself (L1, the paper's default)
    cfg = CF.CFG1_NET
    net = make_net(nv, cfg)
    params = I.uniform_params(net.n_params, seed=9)
    net.set_params(params)
    x = I.uniform_points(2048, seed=10)
    t = np.random.default_rng(11).uniform(size=2048).astype(np.float32)
    # points whose masks and whose sign(y - t) the arithmetic decides
    yo, ym, kink = O.forward_mag(onet(cfg), params, x)
    keep = (kink > FP32_TOL) & (np.abs(yo - t) > FP32_TOL * (ym + np.abs(t)))
    x, t, yo = x[keep], t[keep], yo[keep]
    assert len(t) > 1900
    xt = torch.from_numpy(x).cuda()
    prm = net.parameter()
    y = nv.NeuralVolumeFunction.apply(xt, prm, net)
    loss = (y - torch.from_numpy(t).cuda()).abs().mean()
    loss.backward()
    grads = prm.grad.cpu().numpy().copy()
    dy = np.sign(yo - t) / len(t)
    want = O.backward(onet(cfg), params, x, dy)
    gmag = O.backward_mag(onet(cfg), params, x, np.abs(dy))
    assert mag_err(grads, want, gmag) <= FP32_TOL


# ------------------------------------------------------------- optimizer ----

def test_adam_matches_oracle(nv):
    cfg = CF.CFG1_NET
    net = make_net(nv, cfg)
    params = I.uniform_params(net.n_params, seed=12)
    net.set_params(params)
    net.set_adam(lr=1e-2, l2_reg=1e-6)
    # the hyper-parameters as the ABI carries them (nv_adam_cfg holds floats)
    hp = {k: float(np.float32(v)) for k, v in dict(lr=1e-2, b1=0.9, b2=0.999, eps=1e-15, l2=1e-6).items()}
    rng = np.random.default_rng(13)
    p = params.astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    # magnitudes: p = p0 - sum of the moves; m and v are m and v of the
    # gradient's terms taken by absolute value, |g| + l2 |p|
    pm = np.abs(p).copy()
    q, mm, vv = p.copy(), np.zeros_like(p), np.zeros_like(p)
    for t in range(1, 4):
        g = rng.normal(scale=1e-2, size=net.n_params).astype(np.float32)
        net.buffer("grads").copy_(torch.from_numpy(g).cuda())
        net.optimizer_step()
        before = p.copy()
        O.adam(p, g.astype(np.float64), m, v, t, **hp)
        pm += np.abs(p - before)
        O.adam(q, np.abs(g.astype(np.float64)) + hp["l2"] * np.abs(before), mm, vv, t, **dict(hp, l2=0.0))
    assert mag_err(net.get_params().cpu().numpy(), p, pm) <= FP32_TOL
    assert mag_err(net.buffer("adam_m").cpu().numpy(), m, mm) <= FP32_TOL
    assert mag_err(net.buffer("adam_v").cpu().numpy(), v, vv) <= FP32_TOL
    assert torch.count_nonzero(net.buffer("grads")).item() == 0
    assert net.step_info()[0] == 3


# ---------------------------------------------------------------- sampler ----

def test_sampler_matches_oracle(nv):
    vol = I.blob_volume(32, seed=3)
    vt = torch.from_numpy(vol).cuda()
    for step in (0, 5):
        xyz, t = nv.sample(vt, 10007, seed=99, step=step)
        ox = O.sample_points(99, step, 0, 10007)
        np.testing.assert_array_equal(xyz.cpu().numpy(), ox)
        want = O.trilinear(vol, ox)  # voxels >= 0: the magnitude is the value
        assert mag_err(t.cpu().numpy(), want, want) <= 1e-6


# --------------------------------------------------------------- training ----

def _param_compare(got, want_p, p0, g_oracle, lr):
    """Parameters after Adam: where the oracle gradient is clearly non-zero the
    update is unique and must match (magnitude |p0| + |move|); where it is zero
    up to rounding the sign of the FP32 gradient decides a +-lr step, so only
    validity is checked."""
    got = np.asarray(got, np.float64)
    scale = np.abs(g_oracle).max()
    clear = np.abs(g_oracle) > 1e-4 * scale
    pm = np.abs(p0) + np.abs(want_p - p0)
    assert mag_err(got[clear], want_p[clear], pm[clear]) <= FP32_TOL
    return clear


def test_train_step_cfg2_full_size(nv):
    """One training step of config 2 at full size (2^18 points sampled on the GPU)."""
    cfg = CF.CFG2
    netc = cfg["net"]
    vol = I.blob_volume(cfg["volume"], seed=cfg["volume_seed"])
    vt = torch.from_numpy(vol).cuda()
    net = make_net(nv, netc)
    params = I.init_params(net.n_table, net.n_params - net.n_table, seed=5, dims=netc.dims)
    net.set_params(params)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    n = cfg["batch"]
    net.train_step(n=n, vol=vt, seed=1234, loss_out=loss)
    x = O.sample_points(1234, 0, 0, n)
    t = O.trilinear(vol, x).astype(np.float32)
    tr = O.Trainer(onet(netc), params, lr=cfg["lr"])
    lo = tr.step(x, t)
    assert abs(loss.item() - lo) <= FP32_TOL * lo
    clear = _param_compare(net.get_params().cpu().numpy(), tr.params, params.astype(np.float64), tr.grads,
                           cfg["lr"])
    assert clear.sum() > 0.5 * np.count_nonzero(tr.grads)
    got = net.get_params().cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - params) <= cfg["lr"] * (1 + 1e-4) + 1e-6)


def test_train_trajectory_host_batches(nv):
    """20 steps on host-provided batches: the loss trajectory follows the oracle's."""
    netc = CF.CFG2_NET
    vol = I.blob_volume(32, seed=3)
    net = make_net(nv, netc)
    params = I.init_params(net.n_table, net.n_params - net.n_table, seed=6, dims=netc.dims)
    net.set_params(params)
    tr = O.Trainer(onet(netc), params, lr=1e-2)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    for s in range(20):
        x = O.sample_points(77, s, 0, 4096)
        t = O.trilinear(vol, x).astype(np.float32)
        net.train_step(torch.from_numpy(x), torch.from_numpy(t), loss_out=loss)
        lo = tr.step(x, t)
        # FP32 atomics reorder the gradient sums, and a near-zero gradient's sign
        # then picks a +-lr Adam step, so the tolerance grows with the step count
        assert abs(loss.item() - lo) <= (FP32_TOL + 2e-4 * s) * lo, (s, loss.item(), lo)


# ------------------------------------------------------------- macrocells ----

def test_macrocells_bit_exact(nv):
    vol = I.blob_volume((70, 50, 96), seed=8)
    lut = I.ramp_lut(alpha_floor=0.1)
    mm, mu = nv.macrocells_build(torch.from_numpy(vol).cuda(), 16, torch.from_numpy(lut).cuda())
    omm, omu = O.macrocells(vol, 16, lut)
    np.testing.assert_array_equal(mm.cpu().numpy(), omm)
    np.testing.assert_array_equal(mu.cpu().numpy(), omu)


# --------------------------------------------------------------- rendering ----

def _compare_images(got, want, et=0.99, tol=FP32_TOL):
    """RGBA per pixel against the oracle's (rgba, magnitude) pair: |g - o| <= tol M
    per channel.  A ray that reaches the early-termination opacity may stop one
    sample earlier or later on one side when its opacity is within rounding of
    et; such a pixel moves by at most 1 - et.  Those pixels are allowed that
    bound (and must be rare); every other pixel meets the FP32 tolerance."""
    want, mag = want
    got = got.reshape(-1, 4).astype(np.float64)
    want = want.reshape(-1, 4)
    mag = mag.reshape(-1, 4)
    bad = (np.abs(got - want) > tol * mag).any(axis=1)
    term = np.maximum(got[:, 3], want[:, 3]) >= et - 1e-4
    assert not np.any(bad & ~term), mag_err(got[~term], want[~term], mag[~term])
    straddle = bad & term
    assert straddle.sum() <= max(2, 0.01 * len(want))
    assert np.all(np.abs(got[straddle] - want[straddle]) <= (1 - et) + 1e-4)
    return int(straddle.sum())


def test_render_cfg1_network_full_image(nv):
    cfg = CF.CFG1
    net = make_net(nv, cfg["net"])
    params = I.uniform_params(net.n_params, seed=cfg["param_seed"])
    net.set_params(params)
    W, H = cfg["image"]
    cam = I.ortho_camera_z(W, H)
    lut = I.ramp_lut()
    opts = dict(step=1.0 / cfg["steps"], alpha_exp=1.0, et=0.99, K=8)
    r = nv.Renderer(W * H, K=8)
    img = r.render(cam, torch.from_numpy(lut).cuda(), opts, net=net).cpu().numpy()
    want = O.render_pixels(cam, lut, opts, np.arange(W * H), net=onet(cfg["net"]), params=params, with_mag=True)
    _compare_images(img, want)
    assert want[0][:, 3].max() > 0.1
    it, ns = r.stats()
    assert 0 < it <= cfg["steps"] // 8 + 2


@pytest.mark.parametrize("use_mc", [False, True])
@pytest.mark.parametrize("K", [1, 8])
def test_render_raw_volume_perspective(nv, use_mc, K):
    vol = I.blob_volume(48, seed=4)
    vt = torch.from_numpy(vol).cuda()
    lut = I.ramp_lut(alpha_floor=0.1)
    lt = torch.from_numpy(lut).cuda()
    cam = I.perspective_camera(96, 54)
    opts = dict(step=0.5 / 48, alpha_exp=0.5, et=0.99, K=K, mc_cell=8 if use_mc else 0)
    mc = None
    omu = None
    if use_mc:
        _, mu = nv.macrocells_build(vt, 8, lt)
        mc = (mu, 8, vol.shape)
        omu = O.macrocells(vol, 8, lut)[1]
    r = nv.Renderer(96 * 54, K=K)
    img = r.render(cam, lt, opts, raw=vt, mc=mc).cpu().numpy()
    want = O.render_pixels(cam, lut, opts, np.arange(96 * 54), vol=vol, mumax=omu, with_mag=True)
    _compare_images(img, want)
    assert (want[0][:, 3] > 0).mean() > 0.3


def test_render_cfg3_sampled_pixels(nv):
    """Config 3 geometry at full size (1080p, 512^3, 16^3 macrocells): the
    network render (FP32) checked on sampled pixels the oracle marches one by one."""
    cfg = CF.CFG3
    D = cfg["volume"]
    vt = I.blob_volume_torch(D, cfg["volume_seed"], "cuda")
    vol = vt.cpu().numpy()
    lut = I.ramp_lut(alpha_floor=cfg["alpha_floor"])
    lt = torch.from_numpy(lut).cuda()
    _, mu = nv.macrocells_build(vt, cfg["cell"], lt)
    net = make_net(nv, cfg["net"])
    params = I.init_params(net.n_table, net.n_params - net.n_table, seed=7, dims=cfg["net"].dims)
    params[: net.n_table] = I.uniform_params(net.n_table, seed=8, scale=0.5)
    net.set_params(params)
    W, H = cfg["image"]
    cam = I.perspective_camera(W, H, cfg["vfov"], cfg["eye"], cfg["target"])
    opts = dict(step=cfg["step_voxels"] / D, alpha_exp=cfg["step_voxels"], et=cfg["et"], K=cfg["K"],
                mc_cell=cfg["cell"])
    r = nv.Renderer(W * H, K=cfg["K"])
    img = r.render(cam, lt, opts, net=net, mc=(mu, cfg["cell"], vol.shape)).cpu().numpy().reshape(-1, 4)
    rng = np.random.default_rng(0)
    pix = rng.choice(W * H, 120, replace=False)
    want = O.render_pixels(cam, lut, opts, pix, net=onet(cfg["net"]), params=params, vol=vol,
                           mumax=mu.cpu().numpy(), with_mag=True)
    _compare_images(img[pix], want)
    raw = r.render(cam, lt, opts, raw=vt, mc=(mu, cfg["cell"], vol.shape)).cpu().numpy().reshape(-1, 4)
    want_raw = O.render_pixels(cam, lut, opts, pix, vol=vol, mumax=mu.cpu().numpy(), with_mag=True)
    _compare_images(raw[pix], want_raw)


# ---------------------------------------------------------------- quality ----

def test_image_and_volume_mse(nv):
    a = torch.rand((37, 53, 4), device="cuda")
    b = torch.rand((37, 53, 4), device="cuda")
    got = nv.image_mse(a, b).item()
    want = O.mse(a[..., :3].cpu().numpy().ravel(), b[..., :3].cpu().numpy().ravel())
    assert abs(got - want) <= 1e-12 * want
    cfg = CF.CFG1_NET
    net = make_net(nv, cfg)
    params = I.uniform_params(net.n_params, seed=14)
    net.set_params(params)
    vol = I.blob_volume((20, 33, 41), seed=5)
    got = net.volume_mse(torch.from_numpy(vol).cuda()).item()
    want = O.volume_mse(onet(cfg), params, vol)
    assert abs(got - want) <= FP32_TOL * want
    assert abs(O.psnr(got) - O.psnr(want)) < 1e-4


# ------------------------------------------------------------ measurement ----

def test_peak_kernels_touch_every_access_in_bounds(nv):
    n16, ops = 1 << 12, 5 * nv.PEAK_OPS_QUANTUM
    buf = torch.zeros((n16, 4), dtype=torch.float32, device="cuda")
    nv.peak_scatter(buf, ops, seed=3)
    torch.cuda.synchronize()
    assert buf.double().sum().item() == 4.0 * ops  # every reduction landed (and only in buf)
    assert (buf[:, 0] == buf[:, 3]).all().item()
    assert (buf[:, 0] > 0).float().mean().item() > 0.99  # the mixer spreads the slots
    sink = torch.zeros(1024, dtype=torch.int32, device="cuda")
    nv.peak_gather(buf, ops, sink, seed=4)
    torch.cuda.synchronize()


def test_fp32_generic_shape_matches_oracle(nv):
    """A network outside the register-blocked FP32 kernel's shapes (hidden widths 32 and 16)
    takes the generic one-point-per-thread kernel: forward and backward against the oracle."""
    cfg = CF.NetCfg(4, 2, 12, 4, 1.6, (8, 32, 16, 1))
    net = make_net(nv, cfg)
    params = I.uniform_params(net.n_params, seed=21, scale=0.5)
    net.set_params(params)
    x = I.uniform_points(3000 + 17, seed=22)
    got = net.infer(torch.from_numpy(x).cuda()).cpu().numpy()
    want, wmag, _ = O.forward_mag(onet(cfg), params, x)
    assert mag_err(got, want, wmag) <= FP32_TOL
    x = x[kink_free(onet(cfg), params, x)]
    dy = np.random.default_rng(23).normal(size=x.shape[0]).astype(np.float32)
    g = torch.zeros(net.n_params, dtype=torch.float32, device="cuda")
    net.backward(torch.from_numpy(x).cuda(), torch.from_numpy(dy).cuda(), g)
    want = O.backward(onet(cfg), params, x, dy.astype(np.float64))
    gmag = O.backward_mag(onet(cfg), params, x, np.abs(dy.astype(np.float64)))
    assert mag_err(g.cpu().numpy(), want, gmag) <= FP32_TOL
