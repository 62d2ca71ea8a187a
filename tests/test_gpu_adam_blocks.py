"""The optimizer's reachable-block list (Adam, App. B settings, without an L2
term): blocks of 128 parameters that hold no weight and no hash slot a cell
corner of a point in [0,1]^3 can map to are not visited.  These tests check
that the list is what an independent enumeration of the grid vertices gives,
that training with it equals dense Adam bit for bit, and that every condition
that could break its premise turns it off for good."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2207_11620_gb300 import configs as CF
from paper_2207_11620_gb300 import inputs as I

pytestmark = pytest.mark.gpu

BLOCK = 128  # parameters per block: one warp's float4 per lane


@pytest.fixture(scope="module")
def nv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_11620_gb300 import build, nv as nvmod
    build.build()
    return nvmod


def reachable_blocks(L, F, log2T, res, n_params):
    """Blocks Adam must visit, by brute force over the grid vertices (x, y, z in
    0..N+1 covers both corners of every cell of a point in [0,1]^3, the upper
    one included at coordinate 1).  Levels with more than 4 T such vertices are
    counted whole.  Returns a boolean mask over the vectorised blocks."""
    T = 1 << log2T
    n_table = L * T * F
    n4 = n_params // 4
    nblk = -(-n4 // 32)
    on = np.zeros(nblk, bool)
    on[n_table // BLOCK:] = True  # any block holding a weight
    for l in range(L):
        n1 = int(res[l]) + 2
        lo, hi = l * T * F, (l + 1) * T * F
        if n1 ** 3 > 4 * T:
            on[lo // BLOCK:(hi - 1) // BLOCK + 1] = True
            continue
        v = np.arange(n1, dtype=np.uint64)
        x, y, z = np.meshgrid(v, v, v, indexing="ij")
        h = (x ^ ((y * np.uint64(2654435761)) & np.uint64(0xFFFFFFFF))
             ^ ((z * np.uint64(805459861)) & np.uint64(0xFFFFFFFF))) & np.uint64(T - 1)
        on[(lo + h.ravel().astype(np.int64) * F) // BLOCK] = True
    return on


def span_of(mask, n_params):
    """Parameters visited for a block mask: the last block is clipped to the
    vectorised part, the scalar tail (n_params mod 4) is always visited."""
    n4 = n_params // 4
    if mask.sum() > 0.97 * mask.size:
        return n_params
    idx = np.nonzero(mask)[0]
    v = idx.size * BLOCK
    last_end = (int(idx[-1]) + 1) * 32
    if last_end > n4:
        v -= (last_end - n4) * 4
    return v + (n_params - 4 * n4)


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_block_list_matches_vertex_enumeration(nv, prec):
    c = CF.CFG2_NET
    net = nv.NeuralVolume(prec=prec, **c.kwargs())
    mask = reachable_blocks(c.L, c.F, c.log2T, net.res, net.n_params)
    want = span_of(mask, net.n_params)
    assert net.adam_span() == want
    # config 2's coarse levels leave about 4.4 levels' worth of blocks out
    assert net.n_params - want > 4 * (1 << c.log2T) * c.F


def one_point_batches(k, seed):
    """k single-point batches inside [0,1]^3, one of them on the upper faces."""
    x = O.sample_points(seed, 0, 0, k).astype(np.float32)
    x[k // 2] = (1.0, 1.0, 0.25)
    t = np.linspace(0.1, 0.9, k, dtype=np.float32)
    return x, t


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_skipping_blocks_equals_dense_adam_bit_for_bit(nv, prec):
    """Single-point batches make every gradient deterministic (one contribution
    per slot and step), so the skipping context and a context forced dense (a
    gradient buffer handed out) must end with identical parameters."""
    c = CF.CFG2_NET
    nets = [nv.NeuralVolume(prec=prec, **c.kwargs()) for _ in range(2)]
    params = I.init_params(nets[0].n_table, nets[0].n_params - nets[0].n_table, seed=8, dims=c.dims)
    for net in nets:
        net.set_params(params)
        net.set_adam(lr=1e-2)
    nets[1].buffer("grads")  # forces the dense sweep
    assert nets[0].adam_span() < nets[0].n_params
    assert nets[1].adam_span() == nets[1].n_params
    x, t = one_point_batches(12, seed=41)
    for k in range(len(t)):
        xb = torch.from_numpy(x[k:k + 1].copy()).cuda()
        tb = torch.from_numpy(t[k:k + 1].copy()).cuda()
        for net in nets:
            net.train_step(xb, tb)
    a, b = nets[0].get_params(), nets[1].get_params()
    assert not torch.equal(a, torch.from_numpy(params).cuda())
    assert torch.equal(a, b)
    assert nets[0].adam_span() < nets[0].n_params  # points on the faces keep the list


def test_unvisited_blocks_stay_untouched_after_sampled_training(nv):
    """After sampled training steps, every parameter outside the list still
    has its initial value and zero gradient and moments: no gradient reached a
    block the optimizer does not visit."""
    c = CF.CFG2_NET
    net = nv.NeuralVolume(prec="fp16", **c.kwargs())
    params = I.init_params(net.n_table, net.n_params - net.n_table, seed=9, dims=c.dims)
    net.set_params(params)
    vol = torch.from_numpy(I.blob_volume(32, seed=3)).cuda()
    for s in range(4):
        net.train_step(n=1 << 16, vol=vol, seed=5)
    mask = reachable_blocks(c.L, c.F, c.log2T, net.res, net.n_params)
    off = np.repeat(~mask, BLOCK)[:4 * (net.n_params // 4)]
    off = torch.from_numpy(np.concatenate([off, np.zeros(net.n_params - off.size, bool)])).cuda()
    assert int(off.sum()) > 0
    p = net.get_params()
    assert torch.equal(p[off], torch.from_numpy(params).cuda()[off])
    for name in ("grads", "adam_m", "adam_v"):
        buf = net.buffer(name)
        assert int(torch.count_nonzero(buf[off])) == 0, name
    # the visited part did train
    assert int(torch.count_nonzero(net.buffer("adam_m")[~off])) > 0


def test_point_outside_unit_cube_turns_the_list_off(nv):
    c = CF.CFG2_NET
    net = nv.NeuralVolume(prec="fp16", **c.kwargs())
    before = net.adam_span()
    assert before < net.n_params
    xb = torch.tensor([[0.5, 1.0, 0.0]], device="cuda")
    net.train_step(xb, torch.tensor([0.5], device="cuda"))
    assert net.adam_span() == before
    xb = torch.tensor([[0.5, 1.25, 0.5]], device="cuda")
    net.train_step(xb, torch.tensor([0.5], device="cuda"))
    assert net.adam_span() == net.n_params
    net.train_step(torch.tensor([[0.5, 0.5, 0.5]], device="cuda"), torch.tensor([0.5], device="cuda"))
    assert net.adam_span() == net.n_params  # for good


def test_l2_term_turns_the_list_off_for_good(nv):
    c = CF.CFG2_NET
    net = nv.NeuralVolume(prec="fp32", **c.kwargs())
    assert net.adam_span() < net.n_params
    net.set_adam(l2_reg=1e-6)
    assert net.adam_span() == net.n_params
    net.train_step(torch.tensor([[0.5, 0.5, 0.5]], device="cuda"), torch.tensor([0.5], device="cuda"))
    net.set_adam(l2_reg=0.0)
    assert net.adam_span() == net.n_params


def test_small_table_list_follows_the_same_rule(nv):
    """T = 2^14 (8 levels): 93% of the blocks hold a reachable slot."""
    c = CF.CFG1_NET
    net = nv.NeuralVolume(prec="fp32", **c.kwargs())
    mask = reachable_blocks(c.L, c.F, c.log2T, net.res, net.n_params)
    assert net.adam_span() == span_of(mask, net.n_params)
