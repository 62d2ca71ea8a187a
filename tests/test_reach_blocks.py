"""The reachable-block enumeration the optimizer test compares the library
against, checked on the CPU: every hash slot a corner of a point in [0,1]^3
can reach (points sampled in the cube, on its faces and at its corners) lies
in a block the enumeration keeps, and the blocks it leaves out hold none."""
import numpy as np

import oracle as O
from paper_2207_11620_gb300 import configs as CF
from tests.test_gpu_adam_blocks import BLOCK, reachable_blocks


def test_every_touched_slot_is_in_a_kept_block():
    c = CF.CFG2_NET
    net = O.Net(L=c.L, F=c.F, log2T=c.log2T, Nmin=c.Nmin, b=c.b, dims=c.dims)
    n_params = net.n_table + net.n_weights
    mask = reachable_blocks(c.L, c.F, c.log2T, net.res, n_params)
    rng = np.random.default_rng(7)
    pts = [rng.random((200000, 3), dtype=np.float32)]
    faces = rng.random((3000, 3), dtype=np.float32)
    for a in range(3):
        for v in (0.0, 1.0):
            f = faces.copy()
            f[:, a] = v
            pts.append(f)
    corners = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], np.float32)
    pts.append(corners)
    x = np.concatenate(pts)
    idx = O.hash_indices(net, x).astype(np.int64)  # [n][L][8]
    T, F = net.T, net.F
    for l in range(net.L):
        slots = np.unique(idx[:, l, :])
        blocks = (l * T * F + slots * F) // BLOCK
        assert mask[blocks].all(), l


def test_left_out_blocks_hold_no_reachable_slot_on_a_small_grid():
    """Brute force on a small network: enumerate every vertex 0..N+1 of every
    level directly and compare the set of blocks."""
    net = O.Net(L=4, F=2, log2T=14, Nmin=4, b=1.5, dims=(8, 16, 16, 1))
    n_params = net.n_table + net.n_weights
    mask = reachable_blocks(net.L, net.F, net.log2T, net.res, n_params)
    T, F = net.T, net.F
    want = np.zeros_like(mask)
    want[net.n_table // BLOCK:] = True
    for l, N in enumerate(int(r) for r in net.res):
        for z in range(N + 2):
            for y in range(N + 2):
                for x in range(N + 2):
                    h = (x ^ ((y * 2654435761) & 0xFFFFFFFF) ^ ((z * 805459861) & 0xFFFFFFFF)) & (T - 1)
                    want[(l * T * F + h * F) // BLOCK] = True
    np.testing.assert_array_equal(mask, want)
