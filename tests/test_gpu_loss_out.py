"""Where nv_train_step reports the batch loss: device memory, or pinned host
memory that the step's last kernel writes directly (no copy on the stream);
pageable host memory is refused before anything is enqueued.  The value is the
same either way, and it is the oracle's L2 loss of the batch (Sec. 4)."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
from paper_2207_11620_gb300 import configs as CF, inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_11620_gb300 import build, nv as nvmod
    build.build()
    return nvmod


def _setup(nv, prec):
    c = CF.CFG1_NET
    net = nv.NeuralVolume(prec=prec, **c.kwargs())
    params = I.init_params(net.n_table, net.n_params - net.n_table, seed=3, dims=c.dims)
    net.set_params(params)
    vol = I.blob_volume(32, seed=2)
    x = O.sample_points(9, 0, 0, 4096)
    t = O.trilinear(vol, x).astype(np.float32)
    onet = O.Net(L=c.L, F=c.F, log2T=c.log2T, Nmin=c.Nmin, b=c.b, dims=c.dims)
    want = float(np.mean((O.forward(onet, params, x) - t.astype(np.float64)) ** 2))
    return net, torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), want


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_loss_in_pinned_host_memory_equals_the_device_copy(nv, prec):
    net_d, x, t, want = _setup(nv, prec)
    net_h, _, _, _ = _setup(nv, prec)
    dev = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    host = torch.full((1,), float("nan"), dtype=torch.float64).pin_memory()
    for _ in range(3):  # the same steps on two identical contexts
        net_d.train_step(x, t, loss_out=dev)
        net_h.train_step(x, t, loss_out=host)
    torch.cuda.synchronize()
    assert np.isfinite(host.item())
    # the first step's loss is the oracle's; later steps differ only by the
    # atomics' order, so the two contexts agree to rounding, not bit for bit
    assert host.item() == pytest.approx(dev.item(), rel=1e-5)
    net_h2, _, _, _ = _setup(nv, prec)
    net_h2.train_step(x, t, loss_out=host)
    torch.cuda.synchronize()
    tol = 1e-5 if prec == "fp32" else 2e-2
    assert host.item() == pytest.approx(want, rel=tol)


def test_pageable_host_loss_is_refused(nv):
    net, x, t, _ = _setup(nv, "fp32")
    with pytest.raises(TypeError, match="pinned"):
        net.train_step(x, t, loss_out=torch.zeros(1, dtype=torch.float64))
    # the same through the C ABI: an error status, nothing enqueued
    buf = np.zeros(1, np.float64)
    st = nv.lib().nv_train_step(net.handle, C.c_void_p(x.data_ptr()), C.c_void_p(t.data_ptr()), x.shape[0], None,
                                0, C.c_void_p(buf.ctypes.data))
    assert st == 1 and "pinned host memory" in nv.lib().nv_last_error().decode()
    torch.cuda.synchronize()
    assert buf[0] == 0.0
