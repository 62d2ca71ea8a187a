"""FP64 emulation of the rounding points of the tensor-core MLP (FP16 / BF16
operands, FP32-or-better accumulation), used to derive the gradient
tolerances of the tensor-core path from the arithmetic.

The kernel rounds to the 16-bit type exactly where this model does: the
gathered table entries and the features, the weights W0 and W1, h1, dZ2 and dZ1;
everything else (accumulations, the output layer, the sigmoid, dF and the
weight gradients) stays in FP32 on the GPU and in FP64 here.
"""
import numpy as np

import oracle as O


def round_fp16(a):
    return np.asarray(a, np.float64).astype(np.float16).astype(np.float64)


def round_bf16(a):
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16  # round to nearest even
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


ROUND = {"fp16": round_fp16, "bf16": round_bf16, "exact": lambda a: np.asarray(a, np.float64)}


def backward_model(net: O.Net, params, xyz, dy, prec, scale=128.0):
    """Per-point input gradient dF and the weight gradients (dW0, dW1, dW2) of a
    two-hidden-layer network, with the kernel's rounding points for `prec`."""
    rnd = ROUND[prec]
    p = np.asarray(params, np.float64).copy()
    p[: net.n_table] = rnd(p[: net.n_table])
    d = net.dims
    W = p[net.n_table:]
    W0 = W[: d[1] * d[0]].reshape(d[1], d[0])
    W1 = W[d[1] * d[0]: d[1] * d[0] + d[2] * d[1]].reshape(d[2], d[1])
    W2 = W[-d[2]:]
    f = rnd(O.encode(net, p, xyz))
    z1 = f @ rnd(W0).T
    h1 = rnd(np.maximum(z1, 0))
    z2 = h1 @ rnd(W1).T
    h2 = np.maximum(z2, 0)
    y = 1 / (1 + np.exp(-(h2 @ W2)))
    dz3 = np.asarray(dy, np.float64) * scale * y * (1 - y)
    dZ2 = rnd((dz3[:, None] * W2[None, :]) * (z2 > 0))
    dZ1 = rnd((dZ2 @ rnd(W1)) * (z1 > 0))
    dF = (dZ1 @ rnd(W0)) / scale
    return dF, (dZ1.T @ f) / scale, (dZ2.T @ h1) / scale, (dz3 @ h2) / scale


def forward_model(net: O.Net, params, xyz, prec):
    """Network outputs y with the kernel's rounding points for `prec`."""
    rnd = ROUND[prec]
    p = np.asarray(params, np.float64).copy()
    p[: net.n_table] = rnd(p[: net.n_table])
    d = net.dims
    W = p[net.n_table:]
    W0 = W[: d[1] * d[0]].reshape(d[1], d[0])
    W1 = W[d[1] * d[0]: d[1] * d[0] + d[2] * d[1]].reshape(d[2], d[1])
    W2 = W[-d[2]:]
    f = rnd(O.encode(net, p, xyz))
    h1 = rnd(np.maximum(f @ rnd(W0).T, 0))
    h2 = np.maximum(h1 @ rnd(W1).T, 0)
    return 1 / (1 + np.exp(-(h2 @ W2)))


def table_grad_from_df(net: O.Net, xyz, dF):
    """The table gradient [n_table] of per-point input gradients dF [n][L*F]:
    every cell corner of every level adds its trilinear weight times dF (FP64;
    corner order and cells from the oracle's hash indices and FP32 scaling)."""
    xyz = np.asarray(xyz, np.float32)
    idx = O.hash_indices(net, xyz).astype(np.int64)  # [n][L][8], corner d = dx + 2 dy + 4 dz
    F, T = net.F, net.T
    g = np.zeros(net.n_table)
    for l, N in enumerate(net.res):
        pc = xyz * np.float32(N)  # the kernel's single FP32 multiply
        w = pc.astype(np.float64) - np.floor(pc.astype(np.float64))
        df = dF[:, l * F:(l + 1) * F]
        for d in range(8):
            wt = np.ones(xyz.shape[0])
            for a in range(3):
                wt *= w[:, a] if (d >> a) & 1 else 1.0 - w[:, a]
            slot = (l * T + idx[:, l, d])[:, None] * F + np.arange(F)[None, :]
            np.add.at(g, slot.ravel(), (wt[:, None] * df).ravel())
    return g


def grads_model(net: O.Net, params, xyz, dy, prec, scale=128.0):
    """The whole parameter gradient (tables then W0, W1, W2) with the kernel's
    rounding points for `prec`."""
    dF, dW0, dW1, dW2 = backward_model(net, params, xyz, dy, prec, scale)
    return np.concatenate([table_grad_from_df(net, xyz, dF), dW0.ravel(), dW1.ravel(), np.ravel(dW2)])


def normwise(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def expected_errors(net, params, xyz, dy, prec):
    exact = backward_model(net, params, xyz, dy, "exact")
    got = backward_model(net, params, xyz, dy, prec)
    return {name: normwise(g, e) for name, g, e in zip(("dF", "dW0", "dW1", "dW2"), got, exact)}


def coord_grad_from_df(net: O.Net, params, xyz, dF):
    """dL/dx of every point from a given dL/df: the Jacobian of the trilinear
    encoding (within a cell of level l, d w_a / d x_a = N_l) applied to dF,
    with the unrounded tables (the GPU applies it with its FP32 master tables)."""
    xyz = np.asarray(xyz, np.float32)
    p = np.asarray(params, np.float64)
    idx = O.hash_indices(net, xyz).astype(np.int64)  # [n][L][8], corner d = dx + 2 dy + 4 dz
    n, F, T = xyz.shape[0], net.F, net.T
    g = np.zeros((n, 3))
    for l, N in enumerate(net.res):
        pc = xyz * np.float32(N)  # the kernel's single FP32 multiply
        w = pc.astype(np.float64) - np.floor(pc.astype(np.float64))
        df = dF[:, l * F:(l + 1) * F]
        for d in range(8):
            bits = (d & 1, (d >> 1) & 1, (d >> 2) & 1)
            theta = p[(l * T + idx[:, l, d])[:, None] * F + np.arange(F)[None, :]]
            dot = np.sum(theta * df, axis=1)
            fac = [w[:, a] if bits[a] else 1.0 - w[:, a] for a in range(3)]
            for a in range(3):
                dw = (1.0 if bits[a] else -1.0) * fac[(a + 1) % 3] * fac[(a + 2) % 3]
                g[:, a] += N * dw * dot
    return g
