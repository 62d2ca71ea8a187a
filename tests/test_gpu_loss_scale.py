"""The FP16 loss-scaling branch of the optimizer step (App. B's mixed-precision
training; FP16 static loss scale with overflow skip).

With a loss scale S the FP16 backward multiplies the upstream gradient by S
before the 16-bit products and divides it out again in FP32.  A scale so large
that the 16-bit intermediates overflow (FP16's largest finite value is 65504)
must make the step a no-op: parameters, first and second moments stay bit for
bit as they were, the gradient buffer is cleared, the step is not counted (so
the next step's bias correction and decay schedule are those of the step it
replaces), and S is halved.  Plain FP32 overflow, no GPU fault.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2207_11620_gb300 import configs as CF
from paper_2207_11620_gb300 import inputs as I

pytestmark = pytest.mark.gpu

LR = 1e-2


@pytest.fixture(scope="module")
def nv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_11620_gb300 import build, nv as nvmod
    build.build()
    return nvmod


def onet(c):
    return O.Net(L=c.L, F=c.F, log2T=c.log2T, Nmin=c.Nmin, b=c.b, dims=c.dims)


def _batches():
    vol = I.blob_volume(32, seed=3)
    out = []
    for s in range(2):
        x = O.sample_points(91, s, 0, 4096)
        out.append((x, O.trilinear(vol, x).astype(np.float32)))
    return out


def _net(nvmod, c, params):
    net = nvmod.NeuralVolume(prec="fp16", **c.kwargs())
    net.set_params(params)
    net.set_adam(lr=LR)
    return net


def _state(net):
    return [net.buffer(b).clone() for b in ("params", "adam_m", "adam_v")]


def test_fp16_overflow_skips_the_step_and_halves_the_scale(nv):
    c = CF.CFG1_NET
    (x1, t1), (x2, t2) = _batches()
    on = onet(c)
    params = I.init_params(on.n_table, on.n_weights, seed=17, dims=c.dims)
    net = _net(nv, c, params)
    # the default scale of the FP16 path, and a first ordinary step so that the
    # moments are non-zero before the overflowing one
    assert net.step_info() == (0, 128.0)
    net.train_step(torch.from_numpy(x1), torch.from_numpy(t1))
    net.sync()
    assert net.step_info() == (1, 128.0)
    before = _state(net)
    assert torch.count_nonzero(before[1]).item() > 0

    huge = 3.0e38
    net.set_loss_scale(huge)
    net.train_step(torch.from_numpy(x2), torch.from_numpy(t2))
    net.sync()
    step, scale = net.step_info()
    assert step == 1                       # not counted
    assert scale == np.float32(huge) / 2   # halved on the device
    after = _state(net)
    for name, b, a in zip(("params", "adam_m", "adam_v"), before, after):
        assert torch.equal(b.view(torch.int32), a.view(torch.int32)), name  # bit for bit
    assert torch.count_nonzero(net.buffer("grads")).item() == 0

    # the next step at a sane scale is Adam's second step on batch 2 ...
    net.set_loss_scale(128.0)
    net.train_step(torch.from_numpy(x2), torch.from_numpy(t2))
    net.sync()
    assert net.step_info() == (2, 128.0)
    got = net.get_params().cpu().numpy().astype(np.float64)

    # ... equal to a twin network that never saw the overflow (same two steps);
    # FP32 atomics reorder the gradient sums, so compare where the move is unique
    twin = _net(nv, c, params)
    for x, t in ((x1, t1), (x2, t2)):
        twin.train_step(torch.from_numpy(x), torch.from_numpy(t))
    twin.sync()
    assert twin.step_info() == (2, 128.0)
    ref = twin.get_params().cpu().numpy().astype(np.float64)

    tr = O.Trainer(on, params, lr=LR)
    tr.step(x1, t1)
    g1 = tr.grads.copy()
    tr.step(x2, t2)
    g2 = tr.grads
    clear = (np.abs(g1) > 1e-2 * np.abs(g1).max()) & (np.abs(g2) > 1e-2 * np.abs(g2).max())
    assert clear.sum() > 500
    assert np.max(np.abs(got[clear] - ref[clear])) <= 1e-6
    # and to the oracle's second Adam step (bias corrections of t = 2): 5% noise
    # on both gradients moves a second-step update by < 2% of lr at the 99th
    # percentile, while counting the skipped step (t = 3) moves every one of
    # these by > 5% of lr (median 11%)
    dp_got = got - params
    dp_want = tr.params - params
    agree = np.abs(dp_got[clear] - dp_want[clear]) <= 0.05 * LR
    assert agree.mean() >= 0.99, agree.mean()
