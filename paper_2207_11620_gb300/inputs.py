"""Seeded synthetic inputs shared by the GPU path, its tests, the bench and the oracle.

This module generates inputs only and holds none of the method's arithmetic:
volumes, network initialisations, point batches, transfer functions and
cameras.  The paper trains on scientific scalar fields normalised to [0, 1]
(Sec. 4); those datasets are not available, so a sum of 32 anisotropic
Gaussian blobs plus uniform noise, min-max normalised, stands in for them.

Recipe (every draw from numpy's PCG64 with the given seed, in this order):
  centres  U[0.1, 0.9]^3       (32 x 3)
  sigmas   U[0.02, 0.15]^3     (32 x 3, axis aligned)
  amps     U[0.5, 1.0]         (32)
  value(x) = sum_b amp_b prod_a exp(-(x_a - c_ba)^2 / (2 s_ba^2)) at voxel
             centres x_a = (i + 0.5) / n_a
  + noise  U[0, 0.05] per voxel, then (v - min) / (max - min), float32.
"""
from __future__ import annotations

import numpy as np

N_BLOBS = 32


def blob_params(seed: int):
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.uniform(0.1, 0.9, size=(N_BLOBS, 3))
    sigmas = rng.uniform(0.02, 0.15, size=(N_BLOBS, 3))
    amps = rng.uniform(0.5, 1.0, size=N_BLOBS)
    return rng, centres, sigmas, amps


def _axis_profiles(n: int, centres_a, sigmas_a):
    x = (np.arange(n, dtype=np.float64) + 0.5) / n
    return np.exp(-((x[None, :] - centres_a[:, None]) ** 2) / (2.0 * sigmas_a[:, None] ** 2))


def blob_volume(n, seed: int = 3, noise: float = 0.05) -> np.ndarray:
    """[nz][ny][nx] float32 volume on the host (n is an int or (nz, ny, nx))."""
    nz, ny, nx = (n, n, n) if np.isscalar(n) else tuple(n)
    rng, c, s, a = blob_params(seed)
    gx = _axis_profiles(nx, c[:, 0], s[:, 0])
    gy = _axis_profiles(ny, c[:, 1], s[:, 1])
    gz = _axis_profiles(nz, c[:, 2], s[:, 2])
    zy = (a[:, None, None] * gz[:, :, None] * gy[:, None, :]).reshape(N_BLOBS, nz * ny)
    v = (zy.T @ gx).reshape(nz, ny, nx).astype(np.float32)
    v += rng.uniform(0.0, noise, size=v.shape).astype(np.float32)
    lo, hi = float(v.min()), float(v.max())
    v -= lo
    v *= np.float32(1.0 / (hi - lo))
    return v


def blob_volume_torch(n: int, seed: int, device, noise: float = 0.05, chunk: int = 64):
    """Same blob field generated slab by slab with torch on `device` (large volumes).

    The noise comes from a torch generator seeded with `seed`, so it differs
    from blob_volume()'s but is reproducible on a given device."""
    import torch
    _, c, s, a = blob_params(seed)
    gx = torch.tensor(_axis_profiles(n, c[:, 0], s[:, 0]), dtype=torch.float32, device=device)
    gy = torch.tensor(_axis_profiles(n, c[:, 1], s[:, 1]), dtype=torch.float32, device=device)
    gz = torch.tensor(_axis_profiles(n, c[:, 2], s[:, 2]), dtype=torch.float32, device=device)
    amp = torch.tensor(a, dtype=torch.float32, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    vol = torch.empty((n, n, n), dtype=torch.float32, device=device)
    for z0 in range(0, n, chunk):
        z1 = min(n, z0 + chunk)
        zy = (amp[:, None, None] * gz[:, z0:z1, None] * gy[:, None, :]).reshape(N_BLOBS, -1)
        slab = (zy.t() @ gx).reshape(z1 - z0, n, n)
        slab += torch.rand(slab.shape, generator=gen, device=device) * noise
        vol[z0:z1] = slab
    lo, hi = vol.min(), vol.max()
    vol -= lo
    vol *= 1.0 / (hi - lo)
    return vol


def uniform_params(n: int, seed: int, scale: float = 0.1) -> np.ndarray:
    """n parameters U(-scale, scale) as float32 (tables then weights)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-scale, scale, size=n).astype(np.float32)


def init_params(n_table: int, n_weights: int, seed: int, table_scale: float = 1e-4,
                dims=None) -> np.ndarray:
    """Training initialisation: tables U(-1e-4, 1e-4), weights Xavier-uniform per layer."""
    rng = np.random.Generator(np.random.PCG64(seed))
    tab = rng.uniform(-table_scale, table_scale, size=n_table)
    ws = []
    for k in range(len(dims) - 1):
        lim = np.sqrt(6.0 / (dims[k] + dims[k + 1]))
        ws.append(rng.uniform(-lim, lim, size=dims[k] * dims[k + 1]))
    return np.concatenate([tab] + ws).astype(np.float32)


def uniform_points(n: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(0.0, 1.0, size=(n, 3)).astype(np.float32)


def ramp_lut(alpha_floor: float = 0.0) -> np.ndarray:
    """256-entry RGBA LUT, entry i = (i/255, i/255, i/255, i/255); alpha is 0 below alpha_floor."""
    r = np.arange(256, dtype=np.float32) / 255.0
    lut = np.stack([r, r, r, r], axis=1).astype(np.float32)
    if alpha_floor > 0:
        lut[r < alpha_floor, 3] = 0.0
    return np.ascontiguousarray(lut)


def ramp_lut_soft(floor: float = 0.1) -> np.ndarray:
    """256-entry RGBA LUT: colour i/255, opacity 0 up to `floor` and rising linearly
    from there to 1 at entry 255 (no jump at the floor, unlike ramp_lut(alpha_floor))."""
    r = np.arange(256, dtype=np.float32) / 255.0
    a = np.clip((r - np.float32(floor)) / np.float32(1.0 - floor), 0.0, 1.0).astype(np.float32)
    return np.ascontiguousarray(np.stack([r, r, r, a], axis=1).astype(np.float32))


def ortho_camera_z(width: int, height: int) -> dict:
    """Orthographic camera looking along +z over the unit square (pixel centres)."""
    return dict(eye=(0.5, 0.5, -0.5), target=(0.5, 0.5, 0.5), up=(0.0, 1.0, 0.0),
                tan_half_fovy=0.0, ortho_w=1.0, ortho_h=1.0, width=width, height=height)


def perspective_camera(width: int, height: int, vfov_deg: float = 40.0,
                       eye=(0.5, 0.5, -1.0), target=(0.5, 0.5, 0.5), up=(0.0, 1.0, 0.0)) -> dict:
    return dict(eye=eye, target=target, up=up,
                tan_half_fovy=float(np.float32(np.tan(np.radians(vfov_deg) / 2.0))),
                ortho_w=0.0, ortho_h=0.0, width=width, height=height)


def host_bricks(vol: np.ndarray, brick: int) -> np.ndarray:
    """Brick layout of a volume for out-of-core sampling: [nbz*nby*nbx][(B+2)^3],
    brick (bx, by, bz) holding voxels B*b - 1 .. B*b + B per axis (indices
    clamped to the volume: a one-voxel ghost layer), x fastest."""
    nz, ny, nx = vol.shape
    B = brick
    pad = np.pad(vol, 1, mode="edge")
    out = np.empty((nz // B, ny // B, nx // B, B + 2, B + 2, B + 2), np.float32)
    for bz in range(nz // B):
        for by in range(ny // B):
            for bx in range(nx // B):
                out[bz, by, bx] = pad[bz * B: bz * B + B + 2, by * B: by * B + B + 2, bx * B: bx * B + B + 2]
    return out.reshape(-1, (B + 2) ** 3)


def host_bricks_from_device(vol, brick: int):
    """Same layout built on the GPU slab by slab from a CUDA volume into a pinned
    CPU tensor (for volumes too large to pad on the host)."""
    import torch
    nz, ny, nx = vol.shape
    B = brick
    E = B + 2
    out = torch.empty(((nz // B) * (ny // B) * (nx // B), E ** 3), dtype=torch.float32, pin_memory=True)
    iy = torch.clamp(torch.arange(-1, ny + 1, device=vol.device), 0, ny - 1)
    ix = torch.clamp(torch.arange(-1, nx + 1, device=vol.device), 0, nx - 1)
    per_layer = (ny // B) * (nx // B)
    for bz in range(nz // B):
        iz = torch.clamp(torch.arange(bz * B - 1, bz * B + B + 1, device=vol.device), 0, nz - 1)
        slab = vol.index_select(0, iz).index_select(1, iy).index_select(2, ix)  # [E][ny+2][nx+2]
        bricks = slab.unfold(1, E, B).unfold(2, E, B)                            # [E][nby][nbx][E][E]
        bricks = bricks.permute(1, 2, 0, 3, 4).reshape(per_layer, E ** 3)
        out[bz * per_layer:(bz + 1) * per_layer].copy_(bricks)
    return out
