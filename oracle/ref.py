"""ctypes marshalling for the FP64 oracle in ``oracle.c`` (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
legs use this module.  It holds no arithmetic of the method: every function
converts numpy arrays and calls the C routine of the same name.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")


def build_oracle(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Cam(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3),
                ("tan_half_fovy", C.c_float), ("ortho_w", C.c_float), ("ortho_h", C.c_float),
                ("width", C.c_int), ("height", C.c_int)]


class _Opts(C.Structure):
    _fields_ = [("step", C.c_float), ("alpha_exp", C.c_float), ("et", C.c_float),
                ("mc_cell", C.c_int), ("step_max", C.c_float), ("shade", C.c_int),
                ("light", C.c_float * 3), ("ambient", C.c_float)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build_oracle())
        L = _lib
        L.or_num_threads.restype = C.c_int
        L.or_set_threads.argtypes = [C.c_int]
        L.or_level_res.argtypes = [C.c_int, C.c_int, C.c_double, _i32p]
        L.or_hash.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_uint32]
        L.or_hash.restype = C.c_uint32
        L.or_param_count_dense_coarse.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                                  C.c_int, C.c_int, C.c_int]
        L.or_param_count_dense_coarse.restype = C.c_int64
        L.or_hash_indices.argtypes = [C.c_int, C.c_int, _i32p, _f32p, C.c_int64, _u32p]
        L.or_encode.argtypes = [C.c_int, C.c_int, C.c_int, _i32p, _f64p, _f32p, C.c_int64, _f64p]
        L.or_mlp_forward.argtypes = [_i32p, C.c_int, _f64p, _f64p, C.c_int64, _f64p]
        L.or_forward.argtypes = [C.c_int, C.c_int, C.c_int, _i32p, _i32p, C.c_int, _f64p, _f32p,
                                 C.c_int64, _f64p]
        L.or_loss_l2.argtypes = [_f64p, _f32p, C.c_int64]
        L.or_loss_l2.restype = C.c_double
        L.or_loss_l1.argtypes = [_f64p, _f32p, C.c_int64]
        L.or_loss_l1.restype = C.c_double
        L.or_lr_at.argtypes = [C.c_double, C.c_int, C.c_int, C.c_int, C.c_double]
        L.or_lr_at.restype = C.c_double
        L.or_backward.argtypes = [C.c_int, C.c_int, C.c_int, _i32p, _i32p, C.c_int, _f64p, _f32p,
                                  C.c_int64, _f64p, _f64p]
        L.or_backward_x.argtypes = [C.c_int, C.c_int, C.c_int, _i32p, _i32p, C.c_int, _f64p, _f32p,
                                    C.c_int64, _f64p, _f64p]
        L.or_encode_mag.argtypes = [C.c_int, C.c_int, C.c_int, _i32p, _f64p, _f32p, C.c_int64, _f64p]
        L.or_forward_mag.argtypes = [C.c_int, C.c_int, C.c_int, _i32p, _i32p, C.c_int, _f64p, _f32p,
                                     C.c_int64, _f64p, _f64p, _f64p]
        L.or_backward_mag.argtypes = [C.c_int, C.c_int, C.c_int, _i32p, _i32p, C.c_int, _f64p, _f32p,
                                      C.c_int64, _f64p, C.c_int, _f64p]
        L.or_backward_x_mag.argtypes = [C.c_int, C.c_int, C.c_int, _i32p, _i32p, C.c_int, _f64p, _f32p,
                                        C.c_int64, _f64p, C.c_int, _f64p]
        L.or_adam.argtypes = [_f64p, _f64p, _f64p, _f64p, C.c_int64, C.c_int, C.c_double,
                              C.c_double, C.c_double, C.c_double, C.c_double]
        L.or_train_step.argtypes = [C.c_int, C.c_int, C.c_int, _i32p, _i32p, C.c_int, _f64p, _f64p,
                                    _f64p, _f64p, C.c_int64, _f32p, _f32p, C.c_int64, C.c_int,
                                    C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                    C.c_int, C.c_int, C.c_int, C.c_double]
        L.or_train_step.restype = C.c_double
        L.or_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.or_sample_points.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_int64, _f32p]
        L.or_trilinear.argtypes = [_f32p, C.c_int, C.c_int, C.c_int, _f32p, C.c_int64, _f64p]
        L.or_macrocells.argtypes = [_f32p, C.c_int, C.c_int, C.c_int, C.c_int, _f32p, _f32p, _f32p]
        L.or_mc_online_update.argtypes = [_f32p, _f32p, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_int, _f32p]
        L.or_mc_mu.argtypes = [_f32p, C.c_int64, _f32p, _f32p]
        L.or_march_adaptive_step.argtypes = [_f32p, _f32p, C.c_float, C.c_float, C.c_float, C.c_float, _f32p,
                                             C.c_int, C.c_int, C.c_int, C.c_float, C.c_float, C.c_float,
                                             C.POINTER(C.c_float), _f32p, C.POINTER(C.c_float)]
        L.or_march_adaptive_step.restype = C.c_int
        L.or_render_pixels.argtypes = [C.POINTER(_Cam), _f32p, C.POINTER(_Opts), C.c_int, C.c_int,
                                       C.c_int, C.c_int, _i32p, _i32p, C.c_int, C.c_void_p,
                                       C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, _i64p,
                                       C.c_int64, _f64p, C.c_void_p]
        L.or_pixel_ray.argtypes = [C.POINTER(_Cam), C.c_int, C.c_int, _f32p, _f32p, _f32p]
        L.or_pixel_ray.restype = C.c_int
        L.or_box_exit.argtypes = [_f32p, _f32p]
        L.or_pt_flight.argtypes = [_f32p, _f32p, C.c_float, C.c_float, C.c_float, C.c_float, _f32p, C.c_int,
                                   C.c_int, C.c_int, C.c_float, C.c_float, C.c_float, C.POINTER(C.c_float),
                                   C.POINTER(C.c_float)]
        L.or_pt_flight.restype = C.c_int
        L.or_render_pt.argtypes = [C.POINTER(_Cam), _f32p, C.POINTER(_PtOpts), C.c_int, C.c_int, C.c_int, C.c_int,
                                   _i32p, _i32p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                   _f32p, C.c_int, _i64p, C.c_int64, _f64p]
        L.or_box_exit.restype = C.c_float
        L.or_mse.argtypes = [_f64p, _f64p, C.c_int64]
        L.or_mse.restype = C.c_double
        L.or_psnr.argtypes = [C.c_double]
        L.or_psnr.restype = C.c_double
        L.or_volume_mse.argtypes = [C.c_int, C.c_int, C.c_int, _i32p, _i32p, C.c_int, _f64p, _f32p,
                                    C.c_int, C.c_int, C.c_int]
        L.or_volume_mse.restype = C.c_double
        L.or_brick_sample.argtypes = [_f32p, C.c_int, C.c_int, C.c_int, C.c_int, _i32p, C.c_int, C.c_uint64,
                                      C.c_uint32, C.c_int64, _f32p, _f64p]
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Net:
    """Shape of a hash-encoded network: L levels, F features, T = 2^log2T."""
    L: int
    F: int
    log2T: int
    Nmin: int
    b: float
    dims: tuple

    @property
    def T(self) -> int:
        return 1 << self.log2T

    @property
    def res(self) -> np.ndarray:
        return level_res(self.L, self.Nmin, self.b)

    @property
    def n_table(self) -> int:
        return self.L * self.T * self.F

    @property
    def n_weights(self) -> int:
        d = self.dims
        return sum(d[k] * d[k + 1] for k in range(len(d) - 1))

    @property
    def n_params(self) -> int:
        return self.n_table + self.n_weights

    def _dims(self):
        return np.asarray(self.dims, dtype=np.int32)


def num_threads() -> int:
    return lib().or_num_threads()


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def level_res(L, Nmin, b):
    out = np.zeros(L, dtype=np.int32)
    lib().or_level_res(L, Nmin, float(b), out)
    return out


def hash_vertex(vx, vy, vz, T):
    return int(lib().or_hash(int(vx), int(vy), int(vz), int(T)))


def param_count_dense_coarse(L, F, log2T, base, scale, n_neurons, n_hidden, out_pad=16):
    return int(lib().or_param_count_dense_coarse(L, F, log2T, base, float(scale), n_neurons,
                                                 n_hidden, out_pad))


def hash_indices(net: Net, xyz):
    xyz = _f32(xyz)
    n = xyz.shape[0]
    out = np.zeros((n, net.L, 8), dtype=np.uint32)
    lib().or_hash_indices(net.L, net.log2T, net.res, xyz, n, out)
    return out


def encode(net: Net, params, xyz):
    xyz = _f32(xyz)
    n = xyz.shape[0]
    out = np.zeros((n, net.L * net.F), dtype=np.float64)
    lib().or_encode(net.L, net.F, net.log2T, net.res, _f64(params), xyz, n, out)
    return out


def mlp_forward(dims, weights, inputs):
    inputs = _f64(inputs)
    n = inputs.shape[0]
    out = np.zeros(n, dtype=np.float64)
    lib().or_mlp_forward(np.asarray(dims, dtype=np.int32), len(dims), _f64(weights), inputs, n, out)
    return out


def forward(net: Net, params, xyz):
    xyz = _f32(xyz)
    n = xyz.shape[0]
    out = np.zeros(n, dtype=np.float64)
    lib().or_forward(net.L, net.F, net.log2T, net.res, net._dims(), len(net.dims), _f64(params),
                     xyz, n, out)
    return out


def loss_l2(y, t):
    return float(lib().or_loss_l2(_f64(y), _f32(t), len(y)))


def loss_l1(y, t):
    return float(lib().or_loss_l1(_f64(y), _f32(t), len(y)))


def lr_at(lr0, k, start, interval, base):
    """Learning rate of the 0-based optimizer step k under the exponential decay."""
    return float(lib().or_lr_at(lr0, int(k), int(start), int(interval), base))


def backward(net: Net, params, xyz, dL_dy):
    xyz = _f32(xyz)
    g = np.zeros(net.n_params, dtype=np.float64)
    lib().or_backward(net.L, net.F, net.log2T, net.res, net._dims(), len(net.dims), _f64(params),
                      xyz, xyz.shape[0], _f64(dL_dy), g)
    return g


def backward_x(net: Net, params, xyz, dL_dy):
    """dL/dx of every point, [n][3] float64 (the coordinate gradient)."""
    xyz = _f32(xyz)
    out = np.zeros((xyz.shape[0], 3), dtype=np.float64)
    lib().or_backward_x(net.L, net.F, net.log2T, net.res, net._dims(), len(net.dims), _f64(params),
                        xyz, xyz.shape[0], _f64(dL_dy), out)
    return out


def encode_mag(net: Net, params, xyz):
    """Error magnitudes of the encoded features, [n][L*F] (Sum over corners of w |theta|)."""
    xyz = _f32(xyz)
    n = xyz.shape[0]
    out = np.zeros((n, net.L * net.F), dtype=np.float64)
    lib().or_encode_mag(net.L, net.F, net.log2T, net.res, _f64(params), xyz, n, out)
    return out


def forward_mag(net: Net, params, xyz):
    """(y, M(y), kink margin) of every point: the network value, its error
    magnitude and the smallest |z| / M(z) over the hidden units."""
    xyz = _f32(xyz)
    n = xyz.shape[0]
    y, ym, kink = (np.zeros(n, dtype=np.float64) for _ in range(3))
    lib().or_forward_mag(net.L, net.F, net.log2T, net.res, net._dims(), len(net.dims), _f64(params),
                         xyz, n, y, ym, kink)
    return y, ym, kink


def backward_mag(net: Net, params, xyz, dy_mag, masked=True):
    """Error magnitudes of the parameter gradient (laid out like params) for
    upstream gradients of magnitude dy_mag; masked=False counts every ReLU unit."""
    xyz = _f32(xyz)
    g = np.zeros(net.n_params, dtype=np.float64)
    lib().or_backward_mag(net.L, net.F, net.log2T, net.res, net._dims(), len(net.dims), _f64(params),
                          xyz, xyz.shape[0], _f64(dy_mag), int(bool(masked)), g)
    return g


def backward_x_mag(net: Net, params, xyz, dy_mag, masked=True):
    """Error magnitudes of the coordinate gradient, [n][3]."""
    xyz = _f32(xyz)
    out = np.zeros((xyz.shape[0], 3), dtype=np.float64)
    lib().or_backward_x_mag(net.L, net.F, net.log2T, net.res, net._dims(), len(net.dims), _f64(params),
                            xyz, xyz.shape[0], _f64(dy_mag), int(bool(masked)), out)
    return out


def adam(p, g, m, v, t, lr=1e-2, b1=0.9, b2=0.999, eps=1e-15, l2=0.0):
    """In place on p, m, v (float64 arrays)."""
    lib().or_adam(p, _f64(g), m, v, p.shape[0], int(t), lr, b1, b2, eps, l2)


class Trainer:
    """Oracle training state: FP64 params, Adam moments and the step count."""

    def __init__(self, net: Net, params, lr=1e-2, b1=0.9, b2=0.999, eps=1e-15, l2=0.0, loss="l2",
                 decay_start=2000, decay_interval=1000, decay_base=0.99):
        self.net = net
        self.params = _f64(params).copy()
        self.grads = np.zeros_like(self.params)
        self.m = np.zeros_like(self.params)
        self.v = np.zeros_like(self.params)
        self.t = 0
        if loss not in ("l1", "l2"):
            raise ValueError(loss)
        self.hp = (lr, b1, b2, eps, l2, int(loss == "l1"), int(decay_start), int(decay_interval), decay_base)

    def step(self, xyz, target):
        net = self.net
        self.t += 1
        xyz = _f32(xyz)
        return float(lib().or_train_step(net.L, net.F, net.log2T, net.res, net._dims(),
                                         len(net.dims), self.params, self.grads, self.m, self.v,
                                         net.n_params, xyz, _f32(target), xyz.shape[0], self.t,
                                         *self.hp))


def philox4x32_10(ctr, key):
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(np.asarray(ctr, dtype=np.uint32), np.asarray(key, dtype=np.uint32), out)
    return out


def sample_points(seed, step, first, n):
    out = np.zeros((n, 3), dtype=np.float32)
    lib().or_sample_points(int(seed), int(step), int(first), int(n), out)
    return out


def trilinear(vol, xyz):
    vol = _f32(vol)
    nz, ny, nx = vol.shape
    xyz = _f32(xyz)
    out = np.zeros(xyz.shape[0], dtype=np.float64)
    lib().or_trilinear(vol, nx, ny, nz, xyz, xyz.shape[0], out)
    return out


def macrocells(vol, cell, lut):
    vol = _f32(vol)
    nz, ny, nx = vol.shape
    nc = (-(-nz // cell), -(-ny // cell), -(-nx // cell))
    mm = np.zeros(nc + (2,), dtype=np.float32)
    mu = np.zeros(nc, dtype=np.float32)
    lib().or_macrocells(vol, nx, ny, nz, cell, _f32(lut), mm, mu)
    return mm, mu


def march_adaptive(cam: dict, px, py, opts: dict, mumax, shape):
    """The adaptive march of one pixel as a list of (kind, t_before, t_after, pos, e):
    kind 1 = sample, 2 = crossed transparent cell."""
    o = np.zeros(3, np.float32)
    d = np.zeros(3, np.float32)
    t01 = np.zeros(2, np.float32)
    if not lib().or_pixel_ray(C.byref(_cam(cam)), int(px), int(py), o, d, t01):
        return []
    cell = int(opts["mc_cell"])
    nz, ny, nx = shape
    nc = [-(-n // cell) for n in (nx, ny, nz)]
    sc = [np.float32(n) / np.float32(cell) for n in (nx, ny, nz)]
    mu = _f32(mumax)
    t = C.c_float(t01[0])
    e = C.c_float(0.0)
    pos = np.zeros(3, np.float32)
    steps = []
    while True:
        tb = t.value
        r = lib().or_march_adaptive_step(o, d, float(t01[1]), float(opts["step"]), float(opts["step_max"]),
                                         float(opts.get("alpha_exp", 1.0)), mu, nc[0], nc[1], nc[2],
                                         float(sc[0]), float(sc[1]), float(sc[2]), C.byref(t), pos, C.byref(e))
        if r == 0:
            return steps
        steps.append((r, np.float32(tb), np.float32(t.value), pos.copy(), np.float32(e.value)))


def mc_online_empty(shape, cell):
    """Empty online value ranges [ncz, ncy, ncx, 2] (+inf, -inf) for a volume of `shape` (nz, ny, nx)."""
    nc = tuple(-(-n // cell) for n in shape)
    mm = np.empty(nc + (2,), dtype=np.float32)
    mm[..., 0] = np.inf
    mm[..., 1] = -np.inf
    return mm


def mc_online_update(minmax, xyz, val, shape, cell):
    """Grow the ranges `minmax` (in place) with samples xyz [n, 3] of values val [n]."""
    xyz, val = _f32(xyz), _f32(val)
    assert minmax.dtype == np.float32 and minmax.flags.c_contiguous
    nz, ny, nx = shape
    lib().or_mc_online_update(xyz, val, xyz.shape[0], nx, ny, nz, cell, minmax)
    return minmax


def mc_mu(minmax, lut):
    mu = np.zeros(minmax.shape[:-1], dtype=np.float32)
    lib().or_mc_mu(_f32(minmax), mu.size, _f32(lut), mu)
    return mu


def _cam(cam: dict) -> _Cam:
    c = _Cam()
    for k in ("eye", "target", "up"):
        getattr(c, k)[:] = [float(v) for v in cam[k]]
    c.tan_half_fovy = float(cam.get("tan_half_fovy", 0.0))
    c.ortho_w = float(cam.get("ortho_w", 1.0))
    c.ortho_h = float(cam.get("ortho_h", 1.0))
    c.width = int(cam["width"])
    c.height = int(cam["height"])
    return c


def pixel_ray(cam: dict, px, py):
    o = np.zeros(3, np.float32)
    d = np.zeros(3, np.float32)
    t = np.zeros(2, np.float32)
    hit = lib().or_pixel_ray(C.byref(_cam(cam)), int(px), int(py), o, d, t)
    return bool(hit), o, d, t


class _PtOpts(C.Structure):
    _fields_ = [("density", C.c_float), ("light", C.c_float * 3), ("max_bounces", C.c_int),
                ("seed_lo", C.c_uint32), ("seed_hi", C.c_uint32), ("frame", C.c_uint32)]


def _pt_opts(opts: dict) -> _PtOpts:
    seed = int(opts.get("seed", 0))
    return _PtOpts(float(opts["density"]), (C.c_float * 3)(*[float(v) for v in opts["light"]]),
                   int(opts.get("max_bounces", 8)), seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF,
                   int(opts.get("frame", 0)))


def render_pt(cam: dict, lut, opts: dict, pixels, mumax, cell, vol=None, net: Net | None = None, params=None,
              dims=None):
    """Path-traced radiance (FP64) of the listed pixels for one frame: [n, 4] = RGB, hit flag.
    mumax / cell: the macrocell majorants; vol: the raw volume (or dims (nz, ny, nx) with net)."""
    o = _pt_opts(opts)
    pix = np.ascontiguousarray(pixels, dtype=np.int64)
    out = np.zeros((pix.shape[0], 4), dtype=np.float64)
    if vol is not None:
        vol = _f32(vol)
        nz, ny, nx = vol.shape
        volp = vol.ctypes.data
    else:
        nz, ny, nx = dims
        volp = None
    mu = _f32(mumax)
    if net is not None:
        prm = _f64(params)
        lib().or_render_pt(C.byref(_cam(cam)), _f32(lut), C.byref(o), 1, net.L, net.F, net.log2T, net.res,
                           net._dims(), len(net.dims), prm.ctypes.data, volp, nx, ny, nz, mu, int(cell),
                           pix, pix.shape[0], out)
    else:
        z = np.zeros(1, np.int32)
        lib().or_render_pt(C.byref(_cam(cam)), _f32(lut), C.byref(o), 0, 0, 0, 0, z, z, 0, None, volp, nx,
                           ny, nz, mu, int(cell), pix, pix.shape[0], out)
    return out


def pt_flight(o, d, t, t1, tau, density, mumax, shape, cell):
    """One Woodcock flight of the path tracer: (tentative collision t, its cell majorant) or None."""
    nz, ny, nx = shape
    nc = [-(-n // cell) for n in (nx, ny, nz)]
    sc = [np.float32(n) / np.float32(cell) for n in (nx, ny, nz)]
    tc, mc = C.c_float(0), C.c_float(0)
    ok = lib().or_pt_flight(_f32(o), _f32(d), float(t), float(t1), float(tau), float(density), _f32(mumax),
                            nc[0], nc[1], nc[2], float(sc[0]), float(sc[1]), float(sc[2]), C.byref(tc), C.byref(mc))
    return (np.float32(tc.value), np.float32(mc.value)) if ok else None


def box_exit(o, d):
    return float(lib().or_box_exit(_f32(o), _f32(d)))


def render_pixels(cam: dict, lut, opts: dict, pixels, net: Net | None = None, params=None,
                  vol=None, mumax=None, with_mag=False):
    """RGBA (FP64) of the listed pixels; network values if net is given, else the raw volume.

    vol (with its dims) is also needed for macrocell skipping when mc_cell > 0.
    with_mag: also return the error magnitudes of the four channels."""
    o = _Opts()
    o.step = float(opts["step"])
    o.alpha_exp = float(opts.get("alpha_exp", 1.0))
    o.et = float(opts.get("et", 0.99))
    o.mc_cell = int(opts.get("mc_cell", 0))
    o.step_max = float(opts.get("step_max", 0.0))
    o.shade = int(opts.get("shade", 0))
    o.light = (C.c_float * 3)(*[float(v) for v in opts.get("light", (0.0, 0.0, 0.0))])
    o.ambient = float(opts.get("ambient", 0.0))
    if o.step_max > 0 and o.mc_cell <= 0:
        raise ValueError("the adaptive step needs macrocells (mc_cell > 0)")
    pix = np.ascontiguousarray(pixels, dtype=np.int64)
    out = np.zeros((pix.shape[0], 4), dtype=np.float64)
    mag = np.zeros((pix.shape[0], 4), dtype=np.float64) if with_mag else None
    magp = mag.ctypes.data if with_mag else None
    if vol is not None:
        vol = _f32(vol)
        nz, ny, nx = vol.shape
        volp = vol.ctypes.data
    else:
        nz, ny, nx = opts.get("dims", (1, 1, 1))
        volp = None
    mup = None
    if o.mc_cell > 0:
        mumax = _f32(mumax)
        mup = mumax.ctypes.data
    if net is not None:
        prm = _f64(params)
        lib().or_render_pixels(C.byref(_cam(cam)), _f32(lut), C.byref(o), 1, net.L, net.F, net.log2T,
                               net.res, net._dims(), len(net.dims), prm.ctypes.data, volp, nx, ny,
                               nz, mup, pix, pix.shape[0], out, magp)
    else:
        z = np.zeros(1, np.int32)
        lib().or_render_pixels(C.byref(_cam(cam)), _f32(lut), C.byref(o), 0, 0, 0, 0, z, z, 0, None,
                               volp, nx, ny, nz, mup, pix, pix.shape[0], out, magp)
    return (out, mag) if with_mag else out


def mse(a, b):
    a = _f64(a).ravel()
    b = _f64(b).ravel()
    return float(lib().or_mse(a, b, a.shape[0]))


def psnr(m):
    return float(lib().or_psnr(float(m)))


def volume_mse(net: Net, params, vol):
    vol = _f32(vol)
    nz, ny, nx = vol.shape
    return float(lib().or_volume_mse(net.L, net.F, net.log2T, net.res, net._dims(), len(net.dims),
                                     _f64(params), vol, nx, ny, nz))


def brick_sample(vol, brick, slot_brick, seed, step, n):
    """Out-of-core training sample (Sec. 4.1): points and FP64 targets."""
    vol = _f32(vol)
    nz, ny, nx = vol.shape
    sb = np.ascontiguousarray(slot_brick, dtype=np.int32)
    xyz = np.zeros((n, 3), np.float32)
    t = np.zeros(n, np.float64)
    lib().or_brick_sample(vol, nx, ny, nz, int(brick), sb, len(sb), int(seed), int(step), int(n), xyz, t)
    return xyz, t
