"""GPU parity of the tcgen05 tensor-core path (FP16 / BF16 operands, FP32 accumulate)
against the FP64 oracle.

Network outputs: within 2e-2 max abs error of the oracle, the stated bound of
the mixed-precision path.  Everything the path computes is also checked
element by element against an FP64 emulation of the kernel's own rounding
points (tests/precision_model.py: the 16-bit roundings of the gathered table
entries, the features, W0, W1, h1, dZ2 and dZ1, everything else exact), whose
distance from the oracle is the error the 16-bit arithmetic itself makes
(2.3% FP16 / 5.7% BF16 normwise on config 2's table gradient, a ReLU decision
flipped by the rounded forward near z = 0 staying in the per-point dF; pinned
against the oracle by tests/test_precision_model.py).  Against that emulation
the GPU differs only by its FP32 accumulation order and by the few 16-bit
roundings that order tips to the neighbouring value, each at most one 16-bit
unit u16 (2^-11 FP16, 2^-8 BF16) of a term: so per element |g - model| <= 2
u16 M, M the oracle's error magnitude of the element (Sum |terms|, every ReLU
unit counted).  At most MODEL_FRAC of the elements may exceed that (a unit
whose pre-activation the FP32 and FP64 evaluations put on different sides of
zero moves one point's terms by up to their own size), and none may exceed M
itself.  The upstream gradients of these checks have one sign, so the batch
sums do not cancel.  The full training step, which uses the L2 gradient as it
comes, is checked through the Adam step it produces.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2207_11620_gb300 import configs as CF
from paper_2207_11620_gb300 import inputs as I
from tests.precision_model import forward_model, grads_model

pytestmark = pytest.mark.gpu

OUT_TOL = 2e-2
# normwise errors of the rounding points themselves (the model against the
# oracle; tests/test_precision_model.py checks the model stays within them)
GRAD_TOL = {"fp16": 2e-2, "bf16": 5e-2}     # weight gradients (batch sums)
TABLE_TOL = {"fp16": 4e-2, "bf16": 1e-1}    # table gradients (per-point dF, scattered)
U16 = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}
MODEL_K = 2
MODEL_FRAC = 1e-3
SCALE = {"fp16": 128.0, "bf16": 1.0}  # the library's default loss scales


@pytest.fixture(scope="module")
def nv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_11620_gb300 import build, nv as nvmod
    build.build()
    return nvmod


def onet(c):
    return O.Net(L=c.L, F=c.F, log2T=c.log2T, Nmin=c.Nmin, b=c.b, dims=c.dims)


SMALL_F4 = CF.NetCfg(16, 4, 14, 16, 1.38, (64, 64, 64, 1))   # config 4's shape at a small T
SHAPES = {"cfg1": CF.CFG1_NET, "cfg2": CF.CFG2_NET, "f4d64": SMALL_F4}


def norm_rel(g, o):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    return float(np.linalg.norm(g - o) / max(np.linalg.norm(o), 1e-30))


def check_against_model(got, model, mag, prec, what=""):
    """Element by element: |got - model| <= MODEL_K u16 M for all but MODEL_FRAC
    of the elements, and <= M for every one (M: the oracle's error magnitude)."""
    got = np.asarray(got, np.float64)
    d = np.abs(got - model)
    out = d > MODEL_K * U16[prec] * mag
    assert out.mean() <= MODEL_FRAC, (what, int(out.sum()), out.size)
    assert np.all(d <= mag), (what, float(np.max(d - mag)))
    return int(out.sum())


def check_grads(got, want, x, params, dy, c, prec, scale):
    """Weight and table gradients against the rounding model, element by element;
    the normwise distance to the oracle reported alongside."""
    net = onet(c)
    model = grads_model(net, params, x, dy, prec, scale)
    mag = O.backward_mag(net, params, x, np.abs(dy), masked=False)
    nt = net.n_table
    check_against_model(got[nt:], model[nt:], mag[nt:], prec, "weights")
    check_against_model(got[:nt], model[:nt], mag[:nt], prec, "tables")
    # entries no corner reaches are exactly zero on both sides
    assert np.all(got[:nt][want[:nt] == 0] == 0)
    return norm_rel(got[:nt], want[:nt]), norm_rel(got[nt:], want[nt:])


def varied_params(net, c, seed):
    """Tables U(-1, 1) and Xavier-uniform weights: outputs spread over (0, 1)
    with pre-activations of the size a trained network has."""
    p = I.init_params(net.n_table, net.n_params - net.n_table, seed=seed, dims=c.dims)
    p[: net.n_table] = I.uniform_params(net.n_table, seed=seed + 1, scale=1.0)
    return p


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("shape", ["cfg1", "cfg2", "f4d64"])
@pytest.mark.parametrize("init", ["uniform0.1", "varied"])
def test_tc_infer_matches_oracle(nv, prec, shape, init):
    c = SHAPES[shape]
    net = nv.NeuralVolume(prec=prec, **c.kwargs())
    if init == "varied":
        params = varied_params(net, c, 41)
    else:
        params = I.uniform_params(net.n_params, seed=41, scale=0.1)
    net.set_params(params)
    n = 20000 + 77  # several tiles and a ragged tail
    x = I.uniform_points(n, seed=42)
    got = net.infer(torch.from_numpy(x).cuda()).cpu().numpy()
    want, wmag, _ = O.forward_mag(onet(c), params, x)
    err = float(np.max(np.abs(got - want)))
    assert err <= OUT_TOL, err
    check_against_model(got, forward_model(onet(c), params, x, prec), wmag, prec, "y")
    if init == "varied":
        assert np.std(want) > 0.015


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("shape", ["cfg1", "cfg2", "f4d64"])
def test_tc_backward_matches_oracle(nv, prec, shape):
    c = SHAPES[shape]
    net = nv.NeuralVolume(prec=prec, **c.kwargs())
    params = I.uniform_params(net.n_params, seed=43, scale=0.5)
    net.set_params(params)
    n = 5000 + 3
    x = I.uniform_points(n, seed=44)
    dy = np.random.default_rng(45).uniform(0.5, 1.5, size=n).astype(np.float32) / n
    g = torch.zeros(net.n_params, dtype=torch.float32, device="cuda")
    net.backward(torch.from_numpy(x).cuda(), torch.from_numpy(dy).cuda(), g)
    want = O.backward(onet(c), params, x, dy.astype(np.float64))
    got = g.cpu().numpy()
    check_grads(got, want, x, params, dy.astype(np.float64), c, prec, SCALE[prec])


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tc_train_step_cfg2_full_size(nv, prec):
    """One config-2 step (2^18 points sampled on the GPU) with the tensor-core MLP."""
    cfg = CF.CFG2
    c = cfg["net"]
    vol = I.blob_volume(cfg["volume"], seed=cfg["volume_seed"])
    vt = torch.from_numpy(vol).cuda()
    net = nv.NeuralVolume(prec=prec, **c.kwargs())
    params = I.init_params(net.n_table, net.n_params - net.n_table, seed=5, dims=c.dims)
    net.set_params(params)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    n = cfg["batch"]
    net.train_step(n=n, vol=vt, seed=1234, loss_out=loss)
    x = O.sample_points(1234, 0, 0, n)
    t = O.trilinear(vol, x).astype(np.float32)
    tr = O.Trainer(onet(c), params, lr=cfg["lr"])
    lo = tr.step(x, t)
    assert abs(loss.item() - lo) <= OUT_TOL * lo
    # at step 1 Adam moves every parameter by -lr sign(g): compare the moves
    # where the oracle gradient is clearly away from zero
    got = net.get_params().cpu().numpy().astype(np.float64)
    g = tr.grads
    clear = np.abs(g) > 0.05 * np.abs(g).max()
    dp_got = got - params
    dp_want = tr.params - params
    agree = np.abs(dp_got[clear] - dp_want[clear]) <= 1e-5
    assert agree.mean() >= 0.99, agree.mean()
    assert np.all(np.abs(dp_got) <= cfg["lr"] * (1 + 1e-4) + 1e-6)
    step, ls = net.step_info()
    assert step == 1


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tc_backward_over_several_chunks(nv, prec):
    """More points than one chunk of the tensor-core path (2^19): each chunk's
    kernel scatters the coarsest levels into the dense replicas and a fold
    follows it, so the replicas must come back to zero between chunks.  Config
    1's shape keeps the serial oracle within seconds."""
    c = CF.CFG1_NET
    net = nv.NeuralVolume(prec=prec, **c.kwargs())
    params = I.uniform_params(net.n_params, seed=47, scale=0.5)
    net.set_params(params)
    n = (1 << 19) + 2 * 128 + 5  # two chunks and a ragged tail
    x = I.uniform_points(n, seed=48)
    dy = np.random.default_rng(49).uniform(0.5, 1.5, size=n).astype(np.float32) / n
    g = torch.zeros(net.n_params, dtype=torch.float32, device="cuda")
    xt, dt = torch.from_numpy(x).cuda(), torch.from_numpy(dy).cuda()
    net.backward(xt, dt, g)
    want = O.backward(onet(c), params, x, dy.astype(np.float64))
    got = g.cpu().numpy()
    check_grads(got, want, x, params, dy.astype(np.float64), c, prec, SCALE[prec])
    # a second call adds the same gradient again: nothing was left in the replicas
    net.backward(xt, dt, g)
    again = g.cpu().numpy().astype(np.float64) - got
    nt = net.n_table
    mag = O.backward_mag(onet(c), params, x, np.abs(dy.astype(np.float64)), masked=False)
    # the same kernels on the same points: equal up to FP32 reduction order (and the
    # subtraction of the first call's sum)
    assert np.all(np.abs(again - got) <= 1e-5 * (mag + np.abs(got)))


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tc_training_converges_like_fp32(nv, prec):
    c = CF.CFG2_NET
    vol = torch.from_numpy(I.blob_volume(32, seed=3)).cuda()
    losses = {}
    for p in ("fp32", prec):
        net = nv.NeuralVolume(prec=p, **c.kwargs())
        net.set_params(I.init_params(net.n_table, net.n_params - net.n_table, seed=6, dims=c.dims))
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        hist = []
        for s in range(60):
            net.train_step(n=1 << 14, vol=vol, seed=9, loss_out=loss)
            hist.append(loss.item())
        losses[p] = hist
    assert losses[prec][-1] < 0.2 * losses[prec][0]
    assert losses[prec][-1] < 1.5 * losses["fp32"][-1] + 1e-5


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tc_render_and_volume_mse(nv, prec):
    c = CF.CFG1_NET
    net = nv.NeuralVolume(prec=prec, **c.kwargs())
    params = varied_params(net, c, 46)
    net.set_params(params)
    cam = I.ortho_camera_z(48, 40)
    lut = I.ramp_lut()
    opts = dict(step=1 / 128, alpha_exp=1.0, et=0.99, K=8)
    r = nv.Renderer(48 * 40, K=8)
    img = r.render(cam, torch.from_numpy(lut).cuda(), opts, net=net).cpu().numpy().reshape(-1, 4)
    want = O.render_pixels(cam, lut, opts, np.arange(48 * 40), net=onet(c), params=params)
    # per-sample values within 2e-2 keep composited colours within a few 1e-2
    assert np.max(np.abs(img - want)) <= 5e-2
    vol = I.blob_volume((20, 24, 28), seed=5)
    got = net.volume_mse(torch.from_numpy(vol).cuda()).item()
    ref = O.volume_mse(onet(c), params, vol)
    assert abs(got - ref) <= 0.1 * ref + 1e-4
