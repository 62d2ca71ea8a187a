"""GPU parity of the coordinate gradient dL/dx (nv_backward's dxyz output)
against the FP64 oracle, on the FP32 path and the tensor-core path.

FP32: per component |g - o| <= 1e-5 M, M the oracle's error magnitude of the
component (the per-point sum over 8 L corners cancels; M is its Sum |terms|),
on points whose ReLU pre-activations are clear of zero by more than that
bound.  FP16 / BF16: the per-point dL/df comes from the rounded forward and
backward, with the ReLU decisions that rounding flips near z = 0 left in it,
as for the table gradient; it is checked element by element against the FP64
emulation of the kernel's rounding points (tests/precision_model.py), within 2
u16 M for all but 0.1% of the components and within M for all, as the table
gradient in tests/test_gpu_tc.py.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2207_11620_gb300 import configs as CF
from paper_2207_11620_gb300 import inputs as I
from tests.precision_model import backward_model, coord_grad_from_df
from tests.test_gpu_parity import kink_free, mag_err
from tests.test_gpu_tc import SCALE, check_against_model

pytestmark = pytest.mark.gpu

NORM_TOL = {"fp16": 4e-2, "bf16": 1e-1}
SMALL_F4 = CF.NetCfg(16, 4, 14, 16, 1.38, (64, 64, 64, 1))
SHAPES = {"cfg1": CF.CFG1_NET, "cfg2": CF.CFG2_NET, "f4d64": SMALL_F4}


@pytest.fixture(scope="module")
def nv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_11620_gb300 import build, nv as nvmod
    build.build()
    return nvmod


def onet(c):
    return O.Net(L=c.L, F=c.F, log2T=c.log2T, Nmin=c.Nmin, b=c.b, dims=c.dims)


def run(nv, c, prec, params, x, dy):
    net = nv.NeuralVolume(prec=prec, **c.kwargs())
    net.set_params(params)
    dx = torch.full((x.shape[0], 3), float("nan"), device="cuda")
    g = torch.zeros(net.n_params, dtype=torch.float32, device="cuda")
    net.backward(torch.from_numpy(x).cuda(), torch.from_numpy(dy).cuda(), g, dx)
    return net, g, dx.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("shape", ["cfg1", "cfg2"])
def test_fp32_coordinate_gradient_matches_oracle(nv, shape):
    c = SHAPES[shape]
    params = I.uniform_params(onet(c).n_params, seed=51)
    x = I.uniform_points(3000 + 41, seed=52)  # several tiles of the FP32 kernel and a ragged tail
    x = x[kink_free(onet(c), params, x)]
    n = x.shape[0]
    dy = np.random.default_rng(53).normal(size=n).astype(np.float32)
    _, _, got = run(nv, c, "fp32", params, x, dy)
    want = O.backward_x(onet(c), params, x, dy.astype(np.float64))
    mag = O.backward_x_mag(onet(c), params, x, np.abs(dy.astype(np.float64)))
    assert np.all(np.isfinite(got))
    assert mag_err(got, want, mag) <= 1e-5


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("shape", ["cfg1", "cfg2", "f4d64"])
def test_tc_coordinate_gradient_matches_oracle(nv, prec, shape):
    c = SHAPES[shape]
    params = I.uniform_params(onet(c).n_params, seed=54, scale=0.5)
    n = 5000 + 3
    x = I.uniform_points(n, seed=55)
    dy = np.random.default_rng(56).uniform(0.5, 1.5, size=n).astype(np.float32)
    _, _, got = run(nv, c, prec, params, x, dy)
    assert np.all(np.isfinite(got))
    dy64 = dy.astype(np.float64)
    dF = backward_model(onet(c), params, x, dy64, prec, SCALE[prec])[0]
    model = coord_grad_from_df(onet(c), params, x, dF)
    mag = O.backward_x_mag(onet(c), params, x, np.abs(dy64), masked=False)
    check_against_model(got, model, mag, prec, "dL/dx")


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_requesting_the_coordinate_gradient_leaves_the_parameter_gradient(nv, prec):
    c = CF.CFG1_NET
    params = I.uniform_params(onet(c).n_params, seed=57)
    n = 1000
    x = I.uniform_points(n, seed=58)
    dy = np.random.default_rng(59).normal(size=n).astype(np.float32)
    net = nv.NeuralVolume(prec=prec, **c.kwargs())
    net.set_params(params)
    xt, dt = torch.from_numpy(x).cuda(), torch.from_numpy(dy).cuda()
    g1 = torch.zeros(net.n_params, device="cuda")
    g2 = torch.zeros(net.n_params, device="cuda")
    net.backward(xt, dt, g1)
    net.backward(xt, dt, g2, torch.empty((n, 3), device="cuda"))
    # the scatter's atomics make the two sums differ in rounding only
    torch.testing.assert_close(g1, g2, rtol=1e-5, atol=1e-7)


def test_autograd_returns_the_coordinate_gradient(nv):
    c = CF.CFG1_NET
    params = I.uniform_params(onet(c).n_params, seed=60)
    net = nv.NeuralVolume(prec="fp32", **c.kwargs())
    net.set_params(params)
    xs = I.uniform_points(777, seed=61)
    xs = xs[kink_free(onet(c), params, xs)]
    x = torch.from_numpy(xs).cuda().requires_grad_(True)
    y = nv.NeuralVolumeFunction.apply(x, net.parameter(), net)
    (y * y).sum().backward()
    dy = (2 * y.detach()).cpu().numpy().astype(np.float64)
    want = O.backward_x(onet(c), params, xs, dy)
    mag = O.backward_x_mag(onet(c), params, xs, np.abs(dy))
    assert mag_err(x.grad.cpu().numpy(), want, mag) <= 1e-5


def test_points_on_upper_faces_and_empty_batch(nv):
    """x = 1 puts a point on the upper face of every level's last cell (the
    upper corner N_l + 1 with weight 0); n = 0 is a no-op."""
    c = CF.CFG1_NET
    params = I.uniform_params(onet(c).n_params, seed=62)
    x = np.array([[1.0, 0.5, 0.25], [0.0, 1.0, 1.0], [1.0, 1.0, 1.0]], np.float32)
    dy = np.ones(3, np.float32)
    assert np.all(kink_free(onet(c), params, x))
    _, _, got = run(nv, c, "fp32", params, x, dy)
    want = O.backward_x(onet(c), params, x, dy.astype(np.float64))
    assert mag_err(got, want, O.backward_x_mag(onet(c), params, x, np.abs(dy.astype(np.float64)))) <= 1e-5
    net = nv.NeuralVolume(prec="fp32", **c.kwargs())
    empty = torch.empty((0, 3), device="cuda")
    net.backward(empty, torch.empty(0, device="cuda"), None, torch.empty((0, 3), device="cuda"))
