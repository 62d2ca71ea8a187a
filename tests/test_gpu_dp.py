"""The library's side of the data-parallel step on one GPU: two replicas of a
network (two contexts) run nv_train_grad on the two halves of a batch, their
nv_dp_buffers are summed (gradient) and max-reduced (flags) -- here by torch
on the same GPU, standing in for the collective, with nothing waiting on
anything -- and each runs nv_optimizer_step.  The replicas must end identical,
equal to one context's nv_train_step on the whole batch and to the oracle's
step; Adam must keep skipping the unreachable blocks."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2207_11620_gb300 import configs as CF
from paper_2207_11620_gb300 import dp
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


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_two_replicas_on_one_gpu_equal_one_context(nv, prec):
    c = CF.CFG2_NET
    vol = I.blob_volume(32, seed=3)
    on = onet(c)
    params = I.init_params(on.n_table, on.n_weights, seed=6, dims=c.dims)
    reps = [nv.NeuralVolume(prec=prec, **c.kwargs()) for _ in range(2)]
    single = nv.NeuralVolume(prec=prec, **c.kwargs())
    for net in reps + [single]:
        net.set_params(params)
    span0 = single.adam_span()
    tr = O.Trainer(on, params, lr=1e-2)
    clear = np.ones(on.n_params, bool)  # gradient clearly away from zero at every step: unique moves
    n = 8191  # odd: the halves differ by one point
    for s in range(3):
        x = O.sample_points(44, s, 0, n)
        t = O.trilinear(vol, x).astype(np.float32)
        xt, tt = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
        sums = []
        for r, net in enumerate(reps):
            lo, hi = dp.shard(n, r, 2)
            sums.append(net.train_grad(xt[lo:hi], tt[lo:hi], n))
        (g0, f0), (g1, f1) = reps[0].dp_buffers(), reps[1].dp_buffers()
        g = g0 + g1
        f = torch.maximum(f0, f1)
        for gr, fl in ((g0, f0), (g1, f1)):
            gr.copy_(g)
            fl.copy_(f)
        for net in reps:
            net.optimizer_step()
        loss = (sums[0] + sums[1]).item() / n
        ref_loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        single.train_step(xt, tt, loss_out=ref_loss)
        lo = tr.step(x, t)
        clear &= np.abs(tr.grads) > 1e-2 * np.abs(tr.grads).max()
        tol = 1e-5 if prec == "fp32" else 2e-2
        assert abs(loss - lo) <= tol * lo and abs(ref_loss.item() - lo) <= tol * lo
    p0, p1 = reps[0].get_params(), reps[1].get_params()
    assert torch.equal(p0, p1)  # the same sum and the same update on both replicas
    for net in reps:
        assert net.step_info()[0] == 3
        assert net.adam_span() == span0 < net.n_params  # the reachable-block skipping survives
    got = p0.cpu().numpy().astype(np.float64)
    ref = single.get_params().cpu().numpy().astype(np.float64)
    assert clear.sum() > 300
    if prec == "fp32":
        assert np.max(np.abs(got[clear] - tr.params[clear])) <= 1e-6
        assert np.max(np.abs(ref[clear] - tr.params[clear])) <= 1e-6
    # against the one-context step: the same kernels, the gradient summed in two halves
    assert np.max(np.abs(got[clear] - ref[clear])) <= (1e-6 if prec == "fp32" else 1e-4)


def test_train_grad_rejects_a_shard_larger_than_the_batch(nv):
    c = CF.CFG1_NET
    net = nv.NeuralVolume(prec="fp32", **c.kwargs())
    x = torch.rand((10, 3), device="cuda")
    with pytest.raises(nv.NvError, match="n_total"):
        net.train_grad(x, torch.rand(10, device="cuda"), 5)
    s = net.train_grad(x[:0], torch.rand(0, device="cuda"), 5)  # an empty shard is fine
    assert s.item() == 0.0
