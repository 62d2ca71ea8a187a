"""GPU parity of the paper's default training recipe (Sec. 3.1, App. B) against
the oracle: L1 loss, Adam with an L2 regulariser and an exponentially decaying
learning rate, on the FP32 path and the tensor-core path."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2207_11620_gb300 import configs as CF
from paper_2207_11620_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
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


def recipe(start, interval, base):
    return dict(lr=5e-3, l2_reg=1e-6, decay_start=start, decay_interval=interval, decay_base=base)


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_l1_first_step_with_decay_matches_oracle(nv, prec):
    """decay_start = 0 decays the very first step: Adam then moves every
    parameter whose regularised gradient is clearly non-zero by exactly
    lr * base, in the direction the oracle gives."""
    c = CF.CFG2_NET
    vol = I.blob_volume(32, seed=3)
    net = nv.NeuralVolume(prec=prec, **c.kwargs())
    params = I.init_params(net.n_table, net.n_params - net.n_table, seed=6, dims=c.dims)
    net.set_params(params)
    hp = recipe(0, 1000, 0.5)
    net.set_adam(**hp)
    net.set_loss("l1")
    x = O.sample_points(31, 0, 0, 8192)
    t = O.trilinear(vol, x).astype(np.float32)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    net.train_step(torch.from_numpy(x), torch.from_numpy(t), loss_out=loss)
    tr = O.Trainer(onet(c), params, lr=hp["lr"], l2=hp["l2_reg"], loss="l1", decay_start=0,
                   decay_interval=1000, decay_base=0.5)
    lo = tr.step(x, t)
    assert abs(loss.item() - lo) <= (FP32_TOL if prec == "fp32" else OUT_TOL) * lo
    got = net.get_params().cpu().numpy().astype(np.float64)
    p64 = params.astype(np.float64)
    g_reg = tr.grads + hp["l2_reg"] * p64
    clear = np.abs(g_reg) > (1e-4 if prec == "fp32" else 0.05) * np.abs(g_reg).max()
    dp_got, dp_want = got - p64, tr.params - p64
    np.testing.assert_allclose(np.abs(dp_want[clear]), 5e-3 * 0.5, rtol=1e-6)
    agree = np.abs(dp_got[clear] - dp_want[clear]) <= 1e-6
    assert agree.mean() >= (1.0 if prec == "fp32" else 0.99), agree.mean()
    # nothing moves by more than the decayed rate (plus FP32 rounding of p)
    assert np.all(np.abs(dp_got) <= 5e-3 * 0.5 * (1 + 1e-4) + 1e-6)


def test_l1_decay_trajectory_matches_oracle_fp32(nv):
    """Eight FP32 steps with the decay starting at step 3 and halving every
    two steps: the loss follows the oracle step by step."""
    c = CF.CFG2_NET
    vol = I.blob_volume(32, seed=4)
    net = nv.NeuralVolume(prec="fp32", **c.kwargs())
    params = I.init_params(net.n_table, net.n_params - net.n_table, seed=8, dims=c.dims)
    net.set_params(params)
    hp = recipe(3, 2, 0.5)
    net.set_adam(**hp)
    net.set_loss("l1")
    tr = O.Trainer(onet(c), params, lr=hp["lr"], l2=hp["l2_reg"], loss="l1", decay_start=3,
                   decay_interval=2, decay_base=0.5)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    for s in range(8):
        x = O.sample_points(55, s, 0, 4096)
        t = O.trilinear(vol, x).astype(np.float32)
        net.train_step(torch.from_numpy(x), torch.from_numpy(t), loss_out=loss)
        lo = tr.step(x, t)
        assert abs(loss.item() - lo) <= (FP32_TOL + 2e-4 * s) * lo, (s, loss.item(), lo)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_l1_recipe_converges_like_fp32(nv, prec):
    c = CF.CFG2_NET
    vol = torch.from_numpy(I.blob_volume(32, seed=3)).cuda()
    losses = {}
    for p in ("fp32", prec):
        net = nv.NeuralVolume(prec=p, **c.kwargs())
        net.set_params(I.init_params(net.n_table, net.n_params - net.n_table, seed=6, dims=c.dims))
        net.set_adam(**recipe(20, 10, 0.9))
        net.set_loss("l1")
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        hist = []
        for s in range(80):
            net.train_step(n=1 << 14, vol=vol, seed=9, loss_out=loss)
            hist.append(loss.item())
        losses[p] = hist
    assert losses[prec][-1] < 0.3 * losses[prec][0]
    assert losses[prec][-1] < 1.5 * losses["fp32"][-1] + 1e-4


def test_set_loss_and_adam_reject_bad_arguments(nv):
    net = nv.NeuralVolume(prec="fp32", **CF.CFG1_NET.kwargs())
    with pytest.raises(KeyError):
        net.set_loss("huber")
    with pytest.raises(nv.NvError):
        net.set_adam(decay_base=1.5)
    with pytest.raises(nv.NvError):
        net.set_adam(decay_start=-1)
