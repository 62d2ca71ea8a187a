"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks one oracle function against something other than itself:
values the paper prints, hand-derived vectors, closed forms, brute force,
library routines (numpy / scipy) or finite differences.  No GPU needed.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import ndimage

import oracle as O
from paper_2207_11620_gb300 import inputs as I


def _read_table(path):
    rows = []
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


# ------------------------------------------------------------- encoding ----

def test_level_resolutions_exact():
    # N_l = floor(Nmin b^l) in exact rational arithmetic (Sec. 3.1, Fig. 1B)
    for nmin, b, L in [(16, "1.5", 8), (16, "1.38", 16), (4, "2", 10)]:
        want = [math.floor(Fraction(nmin) * Fraction(b) ** l) for l in range(L)]
        assert list(O.level_res(L, nmin, float(b))) == want


def test_param_counts_match_paper(golden_dir):
    rows = _read_table(os.path.join(golden_dir, "paper_param_counts.txt"))
    assert len(rows) == 7
    for name, L, F, t, base, W, h, count in rows:
        got = O.param_count_dense_coarse(int(L), int(F), int(t), int(base), 2.0, int(W), int(h), 16)
        assert got == int(count), name


def test_hash_vertices_golden(golden_dir):
    rows = _read_table(os.path.join(golden_dir, "hash_vertices.txt"))
    for vx, vy, vz, h in rows:
        full = int(h, 16)
        assert O.hash_vertex(int(vx), int(vy), int(vz), 1 << 32 - 1) == full % (1 << 31)
        for log2T in (4, 14, 19, 22):
            assert O.hash_vertex(int(vx), int(vy), int(vz), 1 << log2T) == full % (1 << log2T)


def test_hash_indices_corner_order():
    # corner d = dx + 2 dy + 4 dz of the cell floor(fl32(x N_l)) at every level
    net = O.Net(L=3, F=2, log2T=10, Nmin=4, b=2.0, dims=(6, 8, 1))
    x = np.array([[0.30, 0.55, 0.81]], np.float32)
    idx = O.hash_indices(net, x)
    for l, N in enumerate(net.res):
        c = [math.floor(float(np.float32(x[0, a]) * np.float32(N))) for a in range(3)]
        for d in range(8):
            v = (c[0] + (d & 1), c[1] + ((d >> 1) & 1), c[2] + ((d >> 2) & 1))
            assert idx[0, l, d] == O.hash_vertex(*v, net.T)


def test_encode_at_vertices_returns_table_entries():
    # at a grid vertex the trilinear weights collapse onto one corner
    net = O.Net(L=4, F=2, log2T=12, Nmin=16, b=2.0, dims=(8, 16, 1))
    params = I.uniform_params(net.n_params, seed=11)
    tab = params[: net.n_table].astype(np.float64).reshape(net.L, net.T, net.F)
    rng = np.random.default_rng(0)
    ijk = rng.integers(0, 16, size=(64, 3))
    x = (ijk / 16.0).astype(np.float32)
    f = O.encode(net, params, x)
    for p in range(len(x)):
        for l, N in enumerate(net.res):
            c = ijk[p] * (N // 16)
            h = O.hash_vertex(*c, net.T)
            assert np.array_equal(f[p, l * 2:(l + 1) * 2], tab[l, h])


def test_encode_reproduces_affine_field():
    # trilinear interpolation is exact for affine fields (tiny grid, no collisions)
    net = O.Net(L=1, F=2, log2T=12, Nmin=4, b=2.0, dims=(2, 4, 1))
    N = 4
    tab = np.zeros((net.T, 2))
    used = set()
    a1, a2 = np.array([0.3, -1.2, 0.7]), np.array([2.0, 0.5, -0.25])
    for vx in range(N + 1):
        for vy in range(N + 1):
            for vz in range(N + 1):
                h = O.hash_vertex(vx, vy, vz, net.T)
                assert h not in used
                used.add(h)
                v = np.array([vx, vy, vz], float)
                tab[h] = [a1 @ v + 0.1, a2 @ v - 0.4]
    params = np.concatenate([tab.ravel(), np.zeros(net.n_weights)])
    x = I.uniform_points(500, seed=5)
    f = O.encode(net, params, x)
    p = x.astype(np.float32) * np.float32(N)
    np.testing.assert_allclose(f[:, 0], p.astype(np.float64) @ a1 + 0.1, rtol=0, atol=1e-12)
    np.testing.assert_allclose(f[:, 1], p.astype(np.float64) @ a2 - 0.4, rtol=0, atol=1e-12)


def test_encode_partition_of_unity():
    net = O.Net(L=5, F=2, log2T=10, Nmin=16, b=1.5, dims=(10, 8, 1))
    params = np.concatenate([np.ones(net.n_table), np.zeros(net.n_weights)])
    f = O.encode(net, params, I.uniform_points(300, seed=2))
    np.testing.assert_allclose(f, 1.0, rtol=0, atol=1e-14)


def test_encode_matches_scipy_trilinear():
    # brute force: a random field on a collision-free vertex grid, interpolated
    # by scipy's order-1 map_coordinates at p = x * N
    net = O.Net(L=1, F=1, log2T=16, Nmin=8, b=2.0, dims=(1, 4, 1))
    N = 8
    rng = np.random.default_rng(3)
    field = rng.normal(size=(N + 1, N + 1, N + 1))  # [vx][vy][vz]
    tab = np.zeros(net.T)
    seen = set()
    for vx in range(N + 1):
        for vy in range(N + 1):
            for vz in range(N + 1):
                h = O.hash_vertex(vx, vy, vz, net.T)
                assert h not in seen
                seen.add(h)
                tab[h] = field[vx, vy, vz]
    params = np.concatenate([tab, np.zeros(net.n_weights)])
    x = I.uniform_points(400, seed=9)
    f = O.encode(net, params, x)[:, 0]
    p = (x.astype(np.float32) * np.float32(N)).astype(np.float64)
    want = ndimage.map_coordinates(field, p.T, order=1, mode="nearest")
    np.testing.assert_allclose(f, want, rtol=0, atol=1e-12)


# ------------------------------------------------------------------ MLP ----

def test_mlp_matches_numpy_chain():
    dims = (32, 64, 64, 1)
    rng = np.random.default_rng(1)
    Ws = [rng.uniform(-0.3, 0.3, size=(dims[k + 1], dims[k])) for k in range(3)]
    x = rng.normal(size=(200, 32))
    h = np.maximum(x @ Ws[0].T, 0)
    h = np.maximum(h @ Ws[1].T, 0)
    want = 1.0 / (1.0 + np.exp(-(h @ Ws[2].T)[:, 0]))
    got = O.mlp_forward(dims, np.concatenate([w.ravel() for w in Ws]), x)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=0)


def test_mlp_zero_weights_gives_half():
    net = O.Net(L=8, F=2, log2T=14, Nmin=16, b=1.5, dims=(16, 64, 64, 1))
    params = I.uniform_params(net.n_params, seed=1)
    params[net.n_table:] = 0
    y = O.forward(net, params, I.uniform_points(100, seed=2))
    np.testing.assert_array_equal(y, 0.5)


# -------------------------------------------------------------- backward ----

def _fd_setup():
    net = O.Net(L=3, F=2, log2T=8, Nmin=4, b=1.6, dims=(6, 16, 16, 1))
    params = I.uniform_params(net.n_params, seed=21, scale=0.5).astype(np.float64)
    x = I.uniform_points(24, seed=22)
    dy = np.random.default_rng(23).normal(size=24)
    return net, params, x, dy


def test_backward_matches_finite_differences():
    net, params, x, dy = _fd_setup()
    g = O.backward(net, params, x, dy)

    def objective(p):
        return float(dy @ O.forward(net, p, x))

    rng = np.random.default_rng(5)
    touched = np.flatnonzero(g[: net.n_table])
    pick = np.concatenate([rng.choice(touched, 40, replace=False),
                           net.n_table + rng.choice(net.n_weights, 40, replace=False)])
    eps = 1e-6
    for i in pick:
        p1, p2 = params.copy(), params.copy()
        p1[i] += eps
        p2[i] -= eps
        fd = (objective(p1) - objective(p2)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_backward_directional_derivative():
    net, params, x, dy = _fd_setup()
    g = O.backward(net, params, x, dy)
    d = np.random.default_rng(7).normal(size=net.n_params)
    eps = 1e-6
    fp = float(dy @ O.forward(net, params + eps * d, x))
    fm = float(dy @ O.forward(net, params - eps * d, x))
    assert abs((fp - fm) / (2 * eps) - g @ d) <= 1e-7 * abs(g @ d) + 1e-9


def test_backward_untouched_entries_zero():
    net, params, x, dy = _fd_setup()
    g = O.backward(net, params, x, dy)
    idx = O.hash_indices(net, x)
    touched = np.zeros((net.L, net.T), bool)
    for l in range(net.L):
        touched[l, idx[:, l, :].ravel()] = True
    gt = g[: net.n_table].reshape(net.L, net.T, net.F)
    assert np.all(gt[~touched] == 0)


def _grid_points(n, q, seed, net, h):
    """Points on the 2^-q lattice (x N_l and x +- h then stay exact in FP32 for
    N_l < 2^(24-q)) whose cells at every level are the same at x - h and x + h
    on every axis, so the trilinear weights are linear in x over [x - h, x + h]."""
    rng = np.random.default_rng(seed)
    res = net.res
    out = []
    while len(out) < n:
        x = rng.integers(1, (1 << q) - 1, size=3) / float(1 << q)
        ok = all(np.floor((x - h) * N).tolist() == np.floor((x + h) * N).tolist() for N in res)
        if ok:
            out.append(x)
    return np.array(out, dtype=np.float32)


def _coord_fd(net, params, x, dy, h):
    fd = np.zeros((x.shape[0], 3))
    for a in range(3):
        xp, xm = x.copy(), x.copy()
        xp[:, a] += np.float32(h)
        xm[:, a] -= np.float32(h)
        fd[:, a] = dy * (O.forward(net, params, xp) - O.forward(net, params, xm)) / (2 * h)
    return fd


def test_coordinate_gradient_matches_finite_differences():
    """Non-negative tables and weights keep every ReLU in its linear part, so
    y is smooth in x; within one cell per level the trilinear weights are
    linear, and central differences on an exact FP32 lattice leave only the
    O(h^2) curvature of the sigmoid."""
    net = O.Net(L=4, F=2, log2T=10, Nmin=4, b=1.5, dims=(8, 16, 16, 1))
    params = np.abs(I.uniform_params(net.n_params, seed=31, scale=0.5)).astype(np.float64)
    h = 2.0 ** -15
    x = _grid_points(40, 15, 32, net, h)
    dy = np.random.default_rng(33).normal(size=x.shape[0])
    g = O.backward_x(net, params, x, dy)
    fd = _coord_fd(net, params, x, dy, h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9 * np.abs(fd).max())
    assert np.abs(g).min() > 0  # every axis carries a gradient


def test_coordinate_gradient_at_config1_scale():
    """Config 1's shape (8 levels up to N = 273, T = 2^14 with hash collisions)
    with non-negative parameters (every ReLU linear, so y is smooth): central
    differences agree up to their O((N h)^2) curvature term."""
    net = O.Net(L=8, F=2, log2T=14, Nmin=16, b=1.5, dims=(16, 64, 64, 1))
    params = np.abs(I.uniform_params(net.n_params, seed=34)).astype(np.float64)
    h = 2.0 ** -15
    x = _grid_points(60, 15, 35, net, h)
    dy = np.random.default_rng(37).normal(size=x.shape[0])
    g = O.backward_x(net, params, x, dy)
    fd = _coord_fd(net, params, x, dy, h)
    np.testing.assert_allclose(g, fd, rtol=1e-4, atol=1e-7 * np.abs(fd).max())


def test_coordinate_gradient_of_a_ramp_is_closed_form():
    """A one-level, one-feature network whose table holds the ramp 0.1 i at
    vertex (i, j, k): trilinear interpolation reproduces the ramp exactly,
    f = 0.8 x, and with one hidden unit (weights w_in, w_out > 0, so the ReLU
    is the identity on f >= 0) y = sigmoid(w_out w_in 0.8 x): dy/dx has a
    closed form and dy/dy, dy/dz are zero."""
    net = O.Net(L=1, F=1, log2T=16, Nmin=8, b=1.0, dims=(1, 1, 1))
    T = net.T
    params = np.zeros(net.n_params)
    # table entry of vertex (i, j, k) = 0.1 * i (a ramp in x), via the hash of each vertex
    for i in range(9):
        for j in range(9):
            for k in range(9):
                hsh = (i ^ ((j * 2654435761) & 0xFFFFFFFF) ^ ((k * 805459861) & 0xFFFFFFFF)) & (T - 1)
                params[hsh] = 0.1 * i
    w_in, w_out = 0.7, 1.3
    params[net.n_table:] = [w_in, w_out]
    x = _grid_points(10, 12, 36, net, 2.0 ** -12)
    # the ramp needs no collisions among the 729 vertices in 2^16 slots; check it
    hs = {(i ^ ((j * 2654435761) & 0xFFFFFFFF) ^ ((k * 805459861) & 0xFFFFFFFF)) & (T - 1)
          for i in range(9) for j in range(9) for k in range(9)}
    assert len(hs) == 729
    g = O.backward_x(net, params, x, np.ones(x.shape[0]))
    f = 0.1 * 8 * x[:, 0].astype(np.float64)                # the interpolated ramp
    y = 1.0 / (1.0 + np.exp(-w_out * w_in * f))
    want_x = y * (1 - y) * w_out * w_in * 0.1 * 8            # d/dx of sigmoid(w_out w_in 0.8 x)
    np.testing.assert_allclose(g[:, 0], want_x, rtol=1e-12)
    np.testing.assert_allclose(g[:, 1:], 0.0, atol=1e-15)


# ------------------------------------------------------------------ Adam ----

def test_adam_first_step_is_signed_lr():
    rng = np.random.default_rng(0)
    p0 = rng.normal(size=1000)
    g = rng.normal(size=1000)
    p, m, v = p0.copy(), np.zeros(1000), np.zeros(1000)
    O.adam(p, g, m, v, t=1, lr=1e-2, eps=1e-15)
    # m_hat = g, v_hat = g^2 at t = 1  =>  p1 = p0 - lr g / (|g| + eps)
    np.testing.assert_allclose(p, p0 - 1e-2 * np.sign(g), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-14)


def test_adam_large_eps_and_l2():
    p0 = np.array([0.5, -2.0, 1.0])
    g = np.array([0.2, 0.0, -3.0])
    p, m, v = p0.copy(), np.zeros(3), np.zeros(3)
    O.adam(p, g, m, v, t=1, lr=0.1, eps=1.0, l2=0.0)
    np.testing.assert_allclose(p, p0 - 0.1 * g / (np.abs(g) + 1.0), rtol=1e-14)
    p, m, v = p0.copy(), np.zeros(3), np.zeros(3)
    O.adam(p, np.zeros(3), m, v, t=1, lr=0.1, eps=1e-15, l2=1e-3)
    np.testing.assert_allclose(p, p0 - 0.1 * np.sign(p0), rtol=1e-12)


def test_adam_constant_gradient_stays_signed_lr():
    # with a constant gradient the bias-corrected moments are exactly g and g^2
    p0 = np.array([1.0, 1.0])
    g = np.array([0.25, -4.0])
    p, m, v = p0.copy(), np.zeros(2), np.zeros(2)
    for t in range(1, 6):
        O.adam(p, g, m, v, t=t, lr=1e-2)
    np.testing.assert_allclose(p, p0 - 5e-2 * np.sign(g), rtol=0, atol=1e-12)


def test_train_step_reduces_loss():
    net = O.Net(L=4, F=2, log2T=10, Nmin=4, b=1.5, dims=(8, 16, 16, 1))
    params = I.init_params(net.n_table, net.n_weights, seed=3, dims=net.dims)
    tr = O.Trainer(net, params, lr=1e-2)
    vol = I.blob_volume(16, seed=3)
    losses = []
    for s in range(60):
        x = O.sample_points(7, s, 0, 512)
        losses.append(tr.step(x, O.trilinear(vol, x).astype(np.float32)))
    assert losses[-1] < 0.5 * losses[0]


@pytest.mark.parametrize("start,interval,base", [(2000, 1000, 0.99), (3, 2, 0.5), (0, 1, 0.9), (5, 7, 0.75)])
def test_lr_decay_matches_procedural_schedule(start, interval, base):
    # App. B's schedule run as a procedure: the rate starts at lr0 and is
    # multiplied by `base` when step `start` begins and then every `interval` steps
    lr0, lr = 5e-3, 5e-3
    for k in range(start + 5 * interval + 3):
        if k >= start and (k - start) % interval == 0:
            lr *= base
        assert O.lr_at(lr0, k, start, interval, base) == pytest.approx(lr, rel=1e-13), k


def test_l1_loss_known_values():
    y = np.array([0.5, 0.25, 0.75, 0.125])
    t = np.array([0.25, 0.5, 0.75, 0.0], np.float32)
    assert O.loss_l1(y, t) == pytest.approx((0.25 + 0.25 + 0.0 + 0.125) / 4, rel=1e-15)
    assert O.loss_l2(y, t) == pytest.approx((0.0625 + 0.0625 + 0.0 + 0.015625) / 4, rel=1e-15)


@pytest.mark.parametrize("loss", ["l1", "l2"])
def test_train_step_gradient_matches_finite_differences(loss):
    # with lr = 0 the step leaves the parameters alone and its gradient scratch
    # holds d(loss)/d(params); compare with central differences of the loss
    net, params, x, _ = _fd_setup()
    y0 = O.forward(net, params, x)
    rng = np.random.default_rng(11)
    t = (y0 + rng.choice([-0.05, 0.05], size=y0.shape)).astype(np.float32)  # away from the L1 kink
    tr = O.Trainer(net, params, lr=0.0, loss=loss)
    l0 = tr.step(x, t)
    lossf = O.loss_l1 if loss == "l1" else O.loss_l2
    assert l0 == pytest.approx(lossf(y0, t), rel=1e-14)
    np.testing.assert_array_equal(tr.params, params.astype(np.float64))
    g = tr.grads
    touched = np.flatnonzero(g[: net.n_table])
    pick = np.concatenate([rng.choice(touched, 30, replace=False),
                           net.n_table + rng.choice(net.n_weights, 30, replace=False)])
    eps = 1e-6
    for i in pick:
        p1, p2 = params.astype(np.float64), params.astype(np.float64)
        p1[i] += eps
        p2[i] -= eps
        fd = (lossf(O.forward(net, p1, x), t) - lossf(O.forward(net, p2, x), t)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])) + 1e-10, (i, fd, g[i])


@pytest.mark.parametrize("start,expect_decays", [(0, 1), (1, 0)])
def test_train_step_first_update_uses_decayed_rate(start, expect_decays):
    # Adam's first update moves every parameter with a non-zero gradient by
    # exactly its learning rate; with decay_start = 0 that rate is already lr0 * base
    net, params, x, _ = _fd_setup()
    t = np.full(x.shape[0], 0.9, np.float32)
    tr = O.Trainer(net, params, lr=1e-3, loss="l2", decay_start=start, decay_interval=4, decay_base=0.5)
    tr.step(x, t)
    moved = np.abs(tr.grads) > 1e-6  # eps = 1e-15 then changes the step by < 1e-9 relative
    assert moved.sum() > 500
    step = np.abs(tr.params - params.astype(np.float64))[moved]
    np.testing.assert_allclose(step, 1e-3 * 0.5 ** expect_decays, rtol=1e-9)


# -------------------------------------------------------------- sampling ----

def test_philox_known_answers(golden_dir):
    for row in _read_table(os.path.join(golden_dir, "philox4x32_10_kat.txt")):
        v = [int(t, 16) for t in row]
        assert list(O.philox4x32_10(v[0:4], v[4:6])) == v[6:10]


def test_sample_points_uniform_and_reproducible():
    a = O.sample_points(1234, 0, 0, 200000)
    assert a.min() >= 0.0 and a.max() < 1.0
    assert np.all(np.abs(a.mean(0) - 0.5) < 5e-3)
    np.testing.assert_array_equal(a[1000:1010], O.sample_points(1234, 0, 1000, 10))
    assert not np.array_equal(a[:10], O.sample_points(1234, 1, 0, 10))
    # every coordinate is a multiple of 2^-24 (24 random bits)
    assert np.all((a * 2 ** 24) == np.floor(a * 2 ** 24))


def test_trilinear_at_voxel_centres_and_edges():
    vol = I.blob_volume((6, 5, 8), seed=2)
    nz, ny, nx = vol.shape
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    x = np.stack([(ix + 0.5) / nx, (iy + 0.5) / ny, (iz + 0.5) / nz], -1).reshape(-1, 3)
    got = O.trilinear(vol, x.astype(np.float32))
    np.testing.assert_array_equal(got, vol.ravel().astype(np.float64))
    corner = O.trilinear(vol, np.array([[0, 0, 0], [0.9999999, 0.9999999, 0.9999999]], np.float32))
    assert corner[0] == vol[0, 0, 0] and corner[1] == vol[-1, -1, -1]


def test_trilinear_matches_scipy():
    vol = I.blob_volume(12, seed=4)
    x = I.uniform_points(1000, seed=8)
    got = O.trilinear(vol, x)
    q = (x.astype(np.float32) * np.float32(12) - np.float32(0.5)).astype(np.float64)
    q = np.clip(q, 0, 11)
    want = ndimage.map_coordinates(vol.astype(np.float64), q[:, ::-1].T, order=1, mode="nearest")
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


# ------------------------------------------------------------ macrocells ----

def test_macrocells_brute_force():
    vol = I.blob_volume((37, 20, 45), seed=6)
    lut = I.ramp_lut(alpha_floor=0.1)
    cell = 8
    mm, mu = O.macrocells(vol, cell, lut)
    nz, ny, nx = vol.shape
    for cz in range(mm.shape[0]):
        for cy in range(mm.shape[1]):
            for cx in range(mm.shape[2]):
                sl = tuple(slice(max(0, c * cell - 1), min(n, c * cell + cell + 1))
                           for c, n in ((cz, nz), (cy, ny), (cx, nx)))
                blk = vol[sl]
                assert mm[cz, cy, cx, 0] == blk.min() and mm[cz, cy, cx, 1] == blk.max()
                lo = int(np.floor(np.float32(blk.min()) * np.float32(255)))
                hi = min(255, int(np.ceil(np.float32(blk.max()) * np.float32(255))))
                assert mu[cz, cy, cx] == lut[lo:hi + 1, 3].max()


# -------------------------------------------------------------- renderer ----

def test_online_macrocells_brute_force():
    # ranges grown from samples equal a per-cell min / max computed by grouping
    # the samples with numpy, the cell taken from the sample position
    rng = np.random.default_rng(4)
    shape, cell = (40, 33, 50), 8
    x = rng.random((5000, 3), dtype=np.float32)
    x[:7] = [[0, 0, 0], [1, 1, 1], [0.9999999, 0.5, 0.25], [0.16, 0.16, 0.16], [0.5, 0.5, 0.5],
             [0.0, 0.999, 0.0], [0.3, 0.2, 0.1]]
    v = rng.random(5000, dtype=np.float32)
    mm = O.mc_online_update(O.mc_online_empty(shape, cell), x, v, shape, cell)
    nc = [-(-n // cell) for n in shape[::-1]]  # x, y, z
    idx = np.stack([np.clip(np.floor(x[:, a] * np.float32(shape[2 - a] / cell)).astype(int), 0, nc[a] - 1)
                    for a in range(3)], 1)
    lo = np.full(nc[::-1], np.inf, np.float32)
    hi = np.full(nc[::-1], -np.inf, np.float32)
    np.minimum.at(lo, (idx[:, 2], idx[:, 1], idx[:, 0]), v)
    np.maximum.at(hi, (idx[:, 2], idx[:, 1], idx[:, 0]), v)
    np.testing.assert_array_equal(mm[..., 0], lo)
    np.testing.assert_array_equal(mm[..., 1], hi)


def test_online_macrocell_mu_agrees_with_voxel_ranges_and_bounds_them():
    vol = I.blob_volume((32, 40, 48), seed=6)
    lut = I.ramp_lut(alpha_floor=0.1)
    mm_v, mu_v = O.macrocells(vol, 8, lut)
    # mu from the voxel ranges reproduces the voxel-pass mu exactly
    np.testing.assert_array_equal(O.mc_mu(mm_v, lut), mu_v)
    # samples of the volume: their values lie inside the aproned voxel range of
    # the cell that holds them, so the online mu never exceeds the voxel-pass mu
    x = O.sample_points(3, 0, 0, 20000)
    t = O.trilinear(vol, x).astype(np.float32)
    mm = O.mc_online_update(O.mc_online_empty(vol.shape, 8), x, t, vol.shape, 8)
    filled = np.isfinite(mm[..., 0])
    assert filled.mean() > 0.99
    assert np.all(mm[..., 0][filled] >= mm_v[..., 0][filled])
    assert np.all(mm[..., 1][filled] <= mm_v[..., 1][filled])
    mu = O.mc_mu(mm, lut)
    assert np.all(mu <= mu_v)
    assert np.all(mu[~filled] == 0)


@pytest.mark.parametrize("cell", [4, 16])
@pytest.mark.parametrize("smax_factor", [1.0, 8.0, 64.0])
@pytest.mark.parametrize("persp", [False, True])
def test_adaptive_step_beer_lambert(cell, smax_factor, persp):
    # constant medium: whatever segments the adaptive march cuts, the opacity
    # exponents add up to the path length, A = 1 - (1 - a)^(L / s_ref) and the
    # colour is rgb * A
    n = 32
    v = np.float32(100.0 / 255.0)
    vol = np.full((n, n, n), v, np.float32)
    lut = I.ramp_lut()
    _, mu = O.macrocells(vol, cell, lut)
    s1 = np.float32(0.5 / n)
    opts = dict(step=float(s1), alpha_exp=0.5, et=2.0, mc_cell=cell, step_max=float(s1 * smax_factor))
    cam = I.perspective_camera(9, 7) if persp else I.ortho_camera_z(9, 7)
    pix = np.arange(63)
    got = O.render_pixels(cam, lut, opts, pix, vol=vol, mumax=mu)
    a = float(lut[100, 3])
    for q, p in enumerate(pix):
        hit, o, d, t01 = O.pixel_ray(cam, p % 9, p // 9)
        if not hit:
            assert np.all(got[q] == 0)
            continue
        L = float(t01[1]) - float(t01[0])
        A = 1.0 - (1.0 - a) ** (L * n)  # s_ref = one voxel = 1 / n
        assert got[q, 3] == pytest.approx(A, abs=2e-5), (q, got[q, 3], A)
        assert got[q, 0] == pytest.approx(float(lut[100, 0]) * got[q, 3], rel=1e-5)


def test_adaptive_step_segments_tile_the_ray():
    # brute-force invariants of the segment sequence on a random macrocell grid
    # with transparent cells: contiguous, never across a face, s_bar where the
    # cell and t1 leave room, samples only in non-empty cells
    rng = np.random.default_rng(3)
    shape, cell = (40, 36, 44), 4
    nc = [-(-n // cell) for n in shape]
    mu = rng.random(nc).astype(np.float32)
    mu[rng.random(nc) < 0.4] = 0.0
    s1 = np.float32(0.5 / 44)
    s2 = np.float32(16 * s1)
    opts = dict(step=float(s1), step_max=float(s2), alpha_exp=0.5, mc_cell=cell)
    cam = I.perspective_camera(24, 20, eye=(0.31, 0.62, -0.9))
    sc = [np.float32(n) / np.float32(cell) for n in shape[::-1]]  # x, y, z

    def cell_of(pt):
        return tuple(int(np.clip(np.floor(np.float32(pt[a]) * sc[a]), 0, nc[2 - a] - 1)) for a in range(3))

    n_samples = n_short = n_tiny = 0
    for p in rng.choice(24 * 20, 60, replace=False):
        hit, o, d, t01 = O.pixel_ray(cam, p % 24, p // 24)
        steps = O.march_adaptive(cam, p % 24, p // 24, opts, mu, shape)
        if not hit:
            assert steps == []
            continue
        t = np.float32(t01[0])
        for kind, tb, ta, pos, e in steps:
            assert tb == t and ta > tb
            t = ta
            tiny = s1 * np.float32(0.0009765625)
            start = o + np.float32(tb + tiny) * d
            c = cell_of(start)
            m = mu[c[2], c[1], c[0]]
            seg = np.float32(ta - tb)
            if kind == 2:
                assert m == 0
                continue
            n_samples += 1
            assert m > 0
            q = np.float32(1) - min(m, np.float32(1))
            sbar = max(s1 + (s2 - s1) * q * q, s1)
            assert seg <= sbar + 4 * np.spacing(np.float32(ta))  # seg re-derived from rounded t
            n_tiny += seg <= tiny * np.float32(1.0001)
            if seg > 2 * tiny:
                assert cell_of(pos) == c  # the midpoint stays in the start cell
            assert abs(e - 0.5 * seg / s1) <= 0.5 * 4 * np.spacing(np.float32(ta)) / s1 + 1e-6 * e
            if seg < sbar * (1 - 1e-5) and ta < t01[1] * (1 - 1e-6):
                n_short += 1  # cut by the face: just past the end is another cell
                assert cell_of(o + np.float32(ta + 1e-4 * s1) * d) != c or seg <= s1 / 1024 * 1.01
        assert t >= t01[1]
    assert n_samples > 500 and n_short > 50
    assert n_tiny <= 0.01 * n_samples  # slivers only where a ray clips a cell corner


def test_adaptive_step_without_adaptivity_is_the_midpoint_rule():
    # s2 = s1 and one macrocell over the whole volume: every segment but the
    # last is s1 long, so the samples sit at t0 + (k + 1/2) s1
    shape, cell = (16, 16, 16), 16
    mu = np.ones((1, 1, 1), np.float32)
    s1 = np.float32(1.0 / 64)
    opts = dict(step=float(s1), step_max=float(s1), alpha_exp=1.0, mc_cell=cell)
    cam = I.perspective_camera(5, 5)
    for p in range(25):
        hit, o, d, t01 = O.pixel_ray(cam, p % 5, p // 5)
        steps = O.march_adaptive(cam, p % 5, p // 5, opts, mu, shape)
        if not hit:
            continue
        for k, (kind, tb, ta, pos, e) in enumerate(steps[:-1]):
            tk = np.float64(t01[0]) + (k + 0.5) * np.float64(s1)
            np.testing.assert_allclose(pos, o + tk * d, atol=2e-6)
            assert e == pytest.approx(1.0, rel=1e-5)


def _first_sample_shadow_closed_form(cam, lut, opts, vol, W, H, ambient, light):
    # constant medium, fixed step: the first sample of every ray has the largest
    # contribution, and the shadow march from it towards the light crosses N
    # samples of the same opacity, N = #{k : fl32(fl32(k + 1/2) s) < L}
    n = vol.shape[0]
    a = float(lut[100, 3])
    e = opts["alpha_exp"]
    s = np.float32(opts["step"])
    want = []
    for p in range(W * H):
        hit, o, d, t01 = O.pixel_ray(cam, p % W, p // W)
        ks = np.arange(4 * n, dtype=np.float32)
        tk = np.float32(t01[0]) + (ks + np.float32(0.5)) * s
        M = int(np.count_nonzero(tk < t01[1]))
        A = 1.0 - (1.0 - a) ** (e * M)
        first = o + tk[0] * d
        # distance from the first sample to the unit box along the light, per axis
        Ls = [((1.0 if la > 0 else 0.0) - float(first[ax])) / la for ax, la in enumerate(light) if la != 0]
        L = min(Ls)
        N = int(np.count_nonzero((ks + np.float32(0.5)) * s < np.float32(L)))
        T = (1.0 - a) ** (e * N)
        k = ambient + (1.0 - ambient) * T
        rgb = float(lut[100, 0]) * A
        want.append([rgb * k, rgb * k, rgb * k, A])
    return np.array(want)


@pytest.mark.parametrize("light", [(1.0, 0.0, 0.0), (0.0, -1.0, 0.0), (0.6, 0.0, -0.8)])
def test_single_shot_shadow_constant_medium(light):
    n = 24
    vol = np.full((n, n, n), np.float32(100.0 / 255.0), np.float32)
    lut = I.ramp_lut()
    W, H = 7, 5
    cam = I.ortho_camera_z(W, H)
    opts = dict(step=0.5 / n, alpha_exp=0.5, et=2.0, shade=1, light=light, ambient=0.2)
    got = O.render_pixels(cam, lut, opts, np.arange(W * H), vol=vol)
    want = _first_sample_shadow_closed_form(cam, lut, opts, vol, W, H, 0.2, light)
    np.testing.assert_allclose(got, want, rtol=1e-6, atol=1e-9)
    # the shadow only darkens: the emission-absorption image is the bound
    ea = O.render_pixels(cam, lut, dict(opts, shade=0), np.arange(W * H), vol=vol)
    assert np.all(got[:, :3] <= ea[:, :3] + 1e-12) and np.all(got[:, 3] == ea[:, 3])


def test_single_shot_shadow_empty_volume_casts_nothing():
    vol = np.zeros((16, 16, 16), np.float32)
    lut = I.ramp_lut(alpha_floor=0.1)
    cam = I.perspective_camera(6, 6)
    opts = dict(step=0.5 / 16, alpha_exp=0.5, et=0.99, shade=1, light=(0.0, 1.0, 0.0), ambient=0.3)
    got = O.render_pixels(cam, lut, opts, np.arange(36), vol=vol)
    assert np.all(got == 0)


def test_pt_flight_spends_the_target_optical_thickness():
    # Hofmann's walk: the majorant's optical thickness from the start to the
    # tentative collision equals tau; integrate it independently along the ray
    rng = np.random.default_rng(8)
    shape, cell = (24, 20, 28), 4
    nc = [-(-n // cell) for n in shape]
    mu = rng.random(nc).astype(np.float32)
    mu[rng.random(nc) < 0.3] = 0
    D = 5.0
    sc = [np.float32(n) / np.float32(cell) for n in shape[::-1]]
    n_col = 0
    for trial in range(40):
        o = rng.random(3).astype(np.float32) * np.float32(0.8) + np.float32(0.1)
        d = rng.normal(size=3)
        d = (d / np.linalg.norm(d)).astype(np.float32)
        t1 = O.box_exit(o, d)
        tau = np.float32(rng.exponential())
        r = O.pt_flight(o, d, 0.0, t1, tau, D, mu, shape, cell)
        ts = np.linspace(0.0, t1, 20001)
        mid = (ts[:-1] + ts[1:]) / 2
        pts = o[None, :].astype(np.float64) + mid[:, None] * d[None, :].astype(np.float64)
        idx = [np.clip(np.floor(pts[:, a] * float(sc[a])).astype(int), 0, nc[2 - a] - 1) for a in range(3)]
        maj = D * mu[idx[2], idx[1], idx[0]].astype(np.float64)
        cum = np.concatenate([[0.0], np.cumsum(maj * np.diff(ts))])
        if r is None:
            assert cum[-1] <= tau + 0.02 * max(1.0, tau)
            continue
        n_col += 1
        tc, m = r
        assert 0 <= tc <= t1
        got = np.interp(float(tc), ts, cum)
        assert abs(got - tau) <= 0.02 * max(1.0, tau) + 2 * D * (t1 / 20000), (trial, got, tau)
        # the returned majorant is the one of the collision's cell
        pc = o.astype(np.float64) + (float(tc) - 1e-6) * d
        cc = [int(np.clip(np.floor(pc[a] * float(sc[a])), 0, nc[2 - a] - 1)) for a in range(3)]
        assert m == pytest.approx(D * mu[cc[2], cc[1], cc[0]], rel=1e-6)
    assert n_col > 15


def _pt_slab(albedo_index, D, mu_scale, frames, seed, black=False, bounces=1):
    n = 16
    vol = np.full((n, n, n), np.float32(albedo_index / 255.0), np.float32)
    lut = I.ramp_lut()
    if black:
        lut[:, :3] = 0
    _, mu = O.macrocells(vol, 8, lut)
    cam = I.ortho_camera_z(32, 32)
    out = []
    for f in range(frames):
        opts = dict(density=D, light=(0.0, 0.0, -1.0), max_bounces=bounces, seed=seed, frame=f)
        out.append(O.render_pt(cam, lut, opts, np.arange(32 * 32), mu * np.float32(mu_scale), 8, vol=vol))
    return np.concatenate(out), lut


@pytest.mark.parametrize("mu_scale", [1.0, 3.0])
def test_pt_single_scatter_closed_form(mu_scale):
    # constant medium, camera rays along +z, light back along -z, one bounce:
    # E[L] = a int_0^1 s e^{-s t} e^{-s t} dt = (a / 2)(1 - e^{-2 s}); an inflated
    # majorant (null collisions) must not change the mean
    k = 100
    D = 3.0
    img, lut = _pt_slab(k, D, mu_scale, 6, seed=11)
    a = float(lut[k, 0])
    sig = D * float(lut[k, 3])
    want = 0.5 * a * (1 - np.exp(-2 * sig))
    L = img[:, 0]
    err = L.std() / np.sqrt(L.size)
    assert abs(L.mean() - want) <= 4 * err, (L.mean(), want, err)
    # P(real collision inside the box) = 1 - e^{-s}
    hit = img[:, 3].mean()
    assert abs(hit - (1 - np.exp(-sig))) <= 4 * np.sqrt(hit * (1 - hit) / img.shape[0])


def test_pt_zero_albedo_is_black():
    img, _ = _pt_slab(100, 3.0, 1.0, 1, seed=2, black=True, bounces=8)
    assert img[:, 3].mean() > 0.5  # the medium is hit ...
    assert np.all(img[:, :3] == 0)  # ... but nothing is scattered


def test_pt_more_bounces_add_light():
    one, _ = _pt_slab(200, 3.0, 1.0, 2, seed=4, bounces=1)
    many, _ = _pt_slab(200, 3.0, 1.0, 2, seed=4, bounces=8)
    # the first bounce is the same path in both (same random numbers until then)
    assert np.all(many[:, 0] >= one[:, 0] - 1e-12)
    assert many[:, 0].mean() > 1.05 * one[:, 0].mean()


def test_ortho_rays_through_pixel_centres():
    cam = I.ortho_camera_z(64, 64)
    for px, py in [(0, 0), (17, 40), (63, 63)]:
        hit, o, d, t = O.pixel_ray(cam, px, py)
        assert hit
        assert abs(o[0] - (px + 0.5) / 64) < 1e-6 and abs(o[1] - (1 - (py + 0.5) / 64)) < 1e-6
        assert o[2] == -0.5 and list(d) == [0.0, 0.0, 1.0]
        assert t[0] == 0.5 and t[1] == 1.5


def test_perspective_rays_symmetric():
    cam = I.perspective_camera(192, 108)
    _, _, d0, _ = O.pixel_ray(cam, 10, 20)
    _, _, d1, _ = O.pixel_ray(cam, 181, 20)
    _, _, d2, _ = O.pixel_ray(cam, 10, 87)
    assert abs(d0[0] + d1[0]) < 1e-6 and abs(d0[1] - d1[1]) < 1e-6
    assert abs(d0[1] + d2[1]) < 1e-6
    assert abs(np.linalg.norm(d0) - 1) < 1e-6
    # the half-angle of the top edge matches the vertical field of view
    _, _, dt, _ = O.pixel_ray(cam, 96, 0)
    ang = math.degrees(math.atan2(dt[1], dt[2]))
    assert abs(ang - 20.0 * (1 - 1 / 108)) < 0.3


def _const_volume(v0, n=8):
    return np.full((n, n, n), v0, np.float32)


@pytest.mark.parametrize("alpha", [0.01, 0.03])
def test_constant_slab_beer_lambert(alpha):
    # constant density: A = 1 - (1 - alpha)^(depth / s1) = 1 - exp(-sigma depth),
    # sigma = -ln(1 - alpha) / s1; colour = rgb * A (emission-absorption)
    lut = np.zeros((256, 4), np.float32)
    lut[:, 0], lut[:, 1], lut[:, 2], lut[:, 3] = 0.8, 0.4, 0.2, alpha
    cam = I.ortho_camera_z(4, 4)
    steps = 128
    for s1_steps in (1.0, 2.0):  # s1 = one step, or two steps (alpha_exp = 1/2)
        opts = dict(step=1.0 / steps, alpha_exp=1.0 / s1_steps, et=0.99)
        out = O.render_pixels(cam, lut, opts, np.arange(16), vol=_const_volume(0.5))
        a32 = float(np.float32(alpha))  # the LUT stores alpha in FP32
        sigma = -math.log(1 - a32) / (s1_steps / steps)
        A = 1 - math.exp(-sigma * 1.0)
        np.testing.assert_allclose(out[:, 3], A, rtol=1e-12)
        np.testing.assert_allclose(out[:, :3], np.broadcast_to(lut[0, :3].astype(np.float64) * A, (16, 3)), rtol=1e-12)


def test_early_termination_stops_at_threshold():
    lut = np.zeros((256, 4), np.float32)
    lut[:, :] = 0.2
    cam = I.ortho_camera_z(2, 2)
    out = O.render_pixels(cam, lut, dict(step=1 / 128, alpha_exp=1.0, et=0.99), np.arange(4),
                          vol=_const_volume(0.3))
    keep = 1.0 - float(np.float32(0.2))  # the LUT stores alpha in FP32
    n_stop = math.ceil(math.log(0.01) / math.log(keep))
    np.testing.assert_allclose(out[:, 3], 1 - keep ** n_stop, rtol=1e-12)


def test_zero_density_is_black():
    lut = I.ramp_lut()
    lut[:, 3] = 0
    cam = I.perspective_camera(8, 6)
    out = O.render_pixels(cam, lut, dict(step=1 / 64, alpha_exp=0.5), np.arange(48),
                          vol=I.blob_volume(16, seed=1))
    assert np.all(out == 0)


def test_macrocell_skipping_is_exact_on_raw_volume():
    # skipped cells have zero opacity over their whole (aproned) value range,
    # so skipping must not change a raw-volume render at all
    vol = I.blob_volume(32, seed=4)
    lut = I.ramp_lut(alpha_floor=0.3)
    _, mu = O.macrocells(vol, 8, lut)
    assert (mu == 0).mean() > 0.2
    cam = I.perspective_camera(48, 32)
    pix = np.arange(48 * 32)
    base = dict(step=1 / 64, alpha_exp=0.5, et=0.99)
    a = O.render_pixels(cam, lut, dict(base, mc_cell=0), pix, vol=vol)
    b = O.render_pixels(cam, lut, dict(base, mc_cell=8), pix, vol=vol, mumax=mu)
    np.testing.assert_array_equal(a, b)
    assert a[:, 3].max() > 0.1


# --------------------------------------------------------------- quality ----

def test_psnr_known_values():
    assert O.psnr(0.01) == pytest.approx(20.0, abs=1e-12)
    assert O.psnr(1e-3) == pytest.approx(30.0, abs=1e-12)
    a = np.zeros(1000)
    b = np.full(1000, 0.1)
    assert O.mse(a, b) == pytest.approx(0.01, rel=1e-14)


def test_volume_mse_zero_weights_closed_form():
    net = O.Net(L=4, F=2, log2T=10, Nmin=4, b=1.5, dims=(8, 16, 1))
    params = I.uniform_params(net.n_params, seed=1)
    params[net.n_table:] = 0
    vol = I.blob_volume((5, 7, 6), seed=3)
    want = float(np.mean((0.5 - vol.astype(np.float64)) ** 2))
    assert O.volume_mse(net, params, vol) == pytest.approx(want, rel=1e-13)


# ----------------------------------------------------------- out of core ----

def test_brick_sample_stays_in_its_brick_and_interpolates():
    vol = I.blob_volume(32, seed=9)
    B = 8
    slots = np.array([0, 5, 63, 17], np.int32)  # bricks of the 4x4x4 grid
    xyz, t = O.brick_sample(vol, B, slots, seed=3, step=1, n=4000)
    # every point lies within half a voxel of a voxel centre of one resident brick
    v = xyz * 32 - 0.5
    centre = np.rint(v)
    assert np.all(np.abs(v - centre) <= 0.5 + 1e-5)
    b = (centre[:, 2] // B) * 16 + (centre[:, 1] // B) * 4 + centre[:, 0] // B
    assert set(np.unique(b).astype(int)) <= set(slots.tolist())
    assert len(np.unique(b)) == 4
    # the target is the volume's trilinear value there
    np.testing.assert_array_equal(t, O.trilinear(vol, xyz))
    # jitter spans the voxel: both halves are reached on every axis
    off = v - centre
    assert np.all(off.min(0) < -0.45) and np.all(off.max(0) > 0.45)


def test_brick_sample_uniform_over_slots_and_voxels():
    vol = I.blob_volume(16, seed=1)
    slots = np.arange(8, dtype=np.int32)  # all 2x2x2 bricks of 8^3
    xyz, _ = O.brick_sample(vol, 8, slots, seed=11, step=0, n=80000)
    counts = np.histogramdd(xyz, bins=(2, 2, 2), range=[(0, 1)] * 3)[0].ravel()
    assert np.all(np.abs(counts / 10000 - 1) < 0.05)
