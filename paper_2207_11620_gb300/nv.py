"""Python binding of libnv.so (include/nv.h): argument marshalling only.

Every function here checks tensor devices, dtypes and shapes, passes raw
pointers to the C ABI and raises NvError on a non-zero status.  All
arithmetic runs in the library's CUDA kernels; there is no CPU fallback: if
libnv.so is missing or cannot load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build as _build

LIB_PATH = _build.LIB

NV_FP32, NV_FP16, NV_BF16 = 0, 1, 2
PREC = {"fp32": NV_FP32, "fp16": NV_FP16, "bf16": NV_BF16}
BUF = {"params": 0, "grads": 1, "adam_m": 2, "adam_v": 3}
KCLASS = {"mlp": 0, "adam": 1, "finish": 2, "render": 3, "other": 4, "encode": 5, "scatter": 6}


class NvError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"nv status {status}: {msg}")
        self.status = status


class Volume(C.Structure):
    _fields_ = [("data_dev", C.c_void_p), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int)]


class Camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3),
                ("tan_half_fovy", C.c_float), ("ortho_w", C.c_float), ("ortho_h", C.c_float),
                ("width", C.c_int), ("height", C.c_int)]


class RenderOpts(C.Structure):
    _fields_ = [("step", C.c_float), ("alpha_exp", C.c_float), ("et", C.c_float), ("K", C.c_int),
                ("step_max", C.c_float), ("shade", C.c_int), ("light", C.c_float * 3), ("ambient", C.c_float)]


def render_opts(opts: dict, K: int) -> RenderOpts:
    """nv_render_opts from a dict: step, alpha_exp (1), et (0.99), K, step_max (0 = fixed step),
    shade (0 = emission-absorption, 1 = single-shot shadows), light (unit direction to it), ambient."""
    return RenderOpts(float(opts["step"]), float(opts.get("alpha_exp", 1.0)), float(opts.get("et", 0.99)),
                      int(opts.get("K", K)), float(opts.get("step_max", 0.0)), int(opts.get("shade", 0)),
                      (C.c_float * 3)(*[float(v) for v in opts.get("light", (0.0, 0.0, 0.0))]),
                      float(opts.get("ambient", 0.0)))


class PtOpts(C.Structure):
    _fields_ = [("density", C.c_float), ("light", C.c_float * 3), ("max_bounces", C.c_int),
                ("seed", C.c_uint64), ("frame", C.c_uint32)]


class Macrocells(C.Structure):
    _fields_ = [("mu_max_dev", C.c_void_p), ("cell", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
                ("nz", C.c_int)]


class AdamCfg(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("l2_reg", C.c_float), ("decay_start", C.c_int), ("decay_interval", C.c_int),
                ("decay_base", C.c_float)]


EXPORTS = {
    "nv_create": ([C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.POINTER(C.c_int), C.c_int, C.c_int,
                   C.c_void_p, C.POINTER(C.c_void_p)], C.c_int),
    "nv_destroy": ([C.c_void_p], C.c_int),
    "nv_set_stream": ([C.c_void_p, C.c_void_p], C.c_int),
    "nv_info": ([C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int)], C.c_int),
    "nv_set_params": ([C.c_void_p, C.c_void_p], C.c_int),
    "nv_get_params": ([C.c_void_p, C.c_void_p], C.c_int),
    "nv_buffer_ptr": ([C.c_void_p, C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_int64)], C.c_int),
    "nv_set_adam": ([C.c_void_p, C.POINTER(AdamCfg)], C.c_int),
    "nv_set_loss_scale": ([C.c_void_p, C.c_float], C.c_int),
    "nv_set_loss": ([C.c_void_p, C.c_int], C.c_int),
    "nv_peak_scatter": ([C.c_void_p, C.c_int64, C.c_int64, C.c_uint64, C.c_void_p], C.c_int),
    "nv_peak_gather": ([C.c_void_p, C.c_int64, C.c_int64, C.c_uint64, C.c_void_p, C.c_void_p], C.c_int),
    "nv_render_pt": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                      C.c_void_p], C.c_int),
    "nv_macrocells_reset": ([C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p], C.c_int),
    "nv_macrocells_update": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                              C.c_void_p], C.c_int),
    "nv_macrocells_mu": ([C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p],
                         C.c_int),
    "nv_set_online_macrocells": ([C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int], C.c_int),
    "nv_render_inshader": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
                           C.c_int),
    "nv_get_step": ([C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_float)], C.c_int),
    "nv_adam_span": ([C.c_void_p, C.POINTER(C.c_int64)], C.c_int),
    "nv_hash_indices": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p], C.c_int),
    "nv_encode": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p], C.c_int),
    "nv_infer": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p], C.c_int),
    "nv_backward": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "nv_optimizer_step": ([C.c_void_p], C.c_int),
    "nv_sample": ([C.POINTER(Volume), C.c_int64, C.c_uint64, C.c_uint32, C.c_void_p, C.c_void_p,
                   C.c_void_p], C.c_int),
    "nv_train_step": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(Volume), C.c_uint64,
                       C.c_void_p], C.c_int),
    "nv_train_grad": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p], C.c_int),
    "nv_dp_buffers": ([C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_int64), C.POINTER(C.c_void_p)], C.c_int),
    "nv_macrocells_build": ([C.POINTER(Volume), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
                            C.c_int),
    "nv_renderer_create": ([C.c_int64, C.c_int, C.c_void_p, C.POINTER(C.c_void_p)], C.c_int),
    "nv_renderer_destroy": ([C.c_void_p], C.c_int),
    "nv_render": ([C.c_void_p, C.c_void_p, C.POINTER(Volume), C.POINTER(Camera), C.c_void_p,
                   C.POINTER(Macrocells), C.POINTER(RenderOpts), C.c_void_p], C.c_int),
    "nv_render_rows": ([C.c_void_p, C.c_void_p, C.POINTER(Volume), C.POINTER(Camera), C.c_void_p,
                        C.POINTER(Macrocells), C.POINTER(RenderOpts), C.c_int, C.c_int, C.c_void_p], C.c_int),
    "nv_render_stats": ([C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int64)], C.c_int),
    "nv_render_raw_noalloc": ([C.POINTER(Volume), C.POINTER(Camera), C.c_void_p, C.POINTER(Macrocells),
                               C.POINTER(RenderOpts), C.c_void_p, C.c_void_p], C.c_int),
    "nv_image_mse": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p], C.c_int),
    "nv_volume_mse": ([C.c_void_p, C.POINTER(Volume), C.c_void_p], C.c_int),
    "nv_mse_f64": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p], C.c_int),
    "nv_ooc_create": ([C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64,
                       C.POINTER(C.c_void_p)], C.c_int),
    "nv_ooc_destroy": ([C.c_void_p], C.c_int),
    "nv_ooc_refresh": ([C.c_void_p, C.c_int, C.c_uint64, C.c_void_p], C.c_int),
    "nv_ooc_sample": ([C.c_void_p, C.c_int64, C.c_uint64, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "nv_ooc_slots": ([C.c_void_p, C.POINTER(C.c_int)], C.c_int),
    "nv_ooc_stats": ([C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_double)], C.c_int),
    "nv_profile_enable": ([C.c_void_p, C.c_int], C.c_int),
    "nv_profile_read": ([C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int)], C.c_int),
    "nv_sync": ([C.c_void_p], C.c_int),
    "nv_last_error": ([], C.c_char_p),
}

_lib = None


def lib():
    """Load libnv.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise NvError(-1, f"{LIB_PATH} is missing: run __graft_entry__.build() first")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in EXPORTS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise NvError(status, lib().nv_last_error().decode(errors="replace"))


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, dtype=torch.float32, name="tensor"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _loss_ptr(t):
    """nv_train_step's loss_dev: a CUDA float64 tensor, or a pinned CPU one (the
    step's last kernel writes the loss there), or None."""
    if t is None:
        return C.c_void_p()
    if t.is_cuda:
        return _dev(t, torch.float64, "loss_out")
    if t.dtype != torch.float64 or not t.is_pinned():
        raise TypeError("loss_out must be a CUDA or a pinned CPU float64 tensor")
    return C.c_void_p(t.data_ptr())


def _points(xyz):
    if xyz.dim() != 2 or xyz.shape[1] != 3:
        raise ValueError("points must be [n, 3]")
    return _dev(xyz, name="xyz"), xyz.shape[0]


def volume(vol: torch.Tensor) -> Volume:
    if vol.dim() != 3:
        raise ValueError("volume must be [nz, ny, nx]")
    v = Volume()
    v.data_dev = _dev(vol, name="volume").value
    v.nz, v.ny, v.nx = (int(s) for s in vol.shape)
    return v


def camera(cam: dict) -> Camera:
    c = Camera()
    for k in ("eye", "target", "up"):
        getattr(c, k)[:] = [float(x) for x in cam[k]]
    c.tan_half_fovy = float(cam.get("tan_half_fovy", 0.0))
    c.ortho_w = float(cam.get("ortho_w", 1.0))
    c.ortho_h = float(cam.get("ortho_h", 1.0))
    c.width = int(cam["width"])
    c.height = int(cam["height"])
    return c


class _CudaArray:
    """Wraps a library-owned device pointer for torch.as_tensor (no copy)."""

    def __init__(self, ptr, n, dtype="<f4"):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": dtype, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


class NeuralVolume:
    """One hash-encoded network (nv_ctx): params, Adam state and scratch on the GPU."""

    def __init__(self, L, F, log2T, Nmin, b, dims, prec="fp32", stream=None):
        self.L, self.F, self.log2T, self.Nmin, self.b = L, F, log2T, Nmin, b
        self.dims = tuple(int(d) for d in dims)
        self.prec = PREC[prec] if isinstance(prec, str) else int(prec)
        arr = (C.c_int * len(self.dims))(*self.dims)
        h = C.c_void_p()
        s = C.c_void_p(stream) if stream is not None else _stream()
        _check(lib().nv_create(L, F, log2T, Nmin, float(b), arr, len(self.dims), self.prec, s, C.byref(h)))
        self._h = h
        n_params, n_table = C.c_int64(), C.c_int64()
        res = (C.c_int * L)()
        _check(lib().nv_info(h, C.byref(n_params), C.byref(n_table), res))
        self.n_params, self.n_table = n_params.value, n_table.value
        self.res = list(res)

    def close(self):
        if getattr(self, "_h", None):
            lib().nv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def set_stream(self, stream=None):
        _check(lib().nv_set_stream(self._h, C.c_void_p(stream) if stream is not None else _stream()))

    def set_params(self, params):
        if isinstance(params, torch.Tensor):
            if params.numel() != self.n_params or params.dtype != torch.float32:
                raise ValueError("params must be float32 of length n_params")
            p = params.contiguous()
            _check(lib().nv_set_params(self._h, C.c_void_p(p.data_ptr())))
        else:
            import numpy as np
            a = np.ascontiguousarray(params, dtype=np.float32)
            if a.size != self.n_params:
                raise ValueError("params must have n_params entries")
            _check(lib().nv_set_params(self._h, C.c_void_p(a.ctypes.data)))

    def get_params(self):
        out = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        _check(lib().nv_get_params(self._h, C.c_void_p(out.data_ptr())))
        return out

    def buffer(self, name):
        """A torch view (no copy) of an internal FP32 buffer: params, grads, adam_m, adam_v."""
        p, n = C.c_void_p(), C.c_int64()
        _check(lib().nv_buffer_ptr(self._h, BUF[name], C.byref(p), C.byref(n)))
        return torch.as_tensor(_CudaArray(p.value, n.value), device="cuda")

    def parameter(self):
        """Leaf tensor viewing the FP32 parameters, for NeuralVolumeFunction."""
        if getattr(self, "_param_view", None) is None:
            self._param_view = self.buffer("params").requires_grad_(True)
        return self._param_view

    def set_adam(self, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-15, l2_reg=0.0, decay_start=2000,
                 decay_interval=1000, decay_base=0.99):
        cfg = AdamCfg(lr, beta1, beta2, eps, l2_reg, decay_start, decay_interval, decay_base)
        _check(lib().nv_set_adam(self._h, C.byref(cfg)))

    def set_online_macrocells(self, minmax, shape=None, cell=None):
        """Let every later train_step widen `minmax` (from online_macrocells) with its
        batch; None turns it off.  shape = volume (nz, ny, nx)."""
        if minmax is None:
            _check(lib().nv_set_online_macrocells(self._h, None, 0, 0, 0, 0))
            self._mc = None
            return
        nz, ny, nx = shape
        _check(lib().nv_set_online_macrocells(self._h, _dev(minmax, name="minmax"), int(nx), int(ny), int(nz),
                                              int(cell)))
        self._mc = minmax  # keep it alive while registered

    def set_loss(self, loss):
        """'l2' (default) or 'l1'."""
        _check(lib().nv_set_loss(self._h, {"l2": 0, "l1": 1}[loss]))

    def set_loss_scale(self, s):
        _check(lib().nv_set_loss_scale(self._h, float(s)))

    def step_info(self):
        st, ls = C.c_int(), C.c_float()
        _check(lib().nv_get_step(self._h, C.byref(st), C.byref(ls)))
        return st.value, ls.value

    def adam_span(self):
        """Parameters the next optimizer step visits (all of them once dense)."""
        v = C.c_int64()
        _check(lib().nv_adam_span(self._h, C.byref(v)))
        return v.value

    def hash_indices(self, xyz):
        p, n = _points(xyz)
        out = torch.empty((n, self.L, 8), dtype=torch.int32, device=xyz.device)
        _check(lib().nv_hash_indices(self._h, p, n, C.c_void_p(out.data_ptr())))
        return out

    def encode(self, xyz):
        p, n = _points(xyz)
        out = torch.empty((n, self.L * self.F), dtype=torch.float32, device=xyz.device)
        _check(lib().nv_encode(self._h, p, n, C.c_void_p(out.data_ptr())))
        return out

    def infer(self, xyz, out=None):
        p, n = _points(xyz)
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device=xyz.device)
        _check(lib().nv_infer(self._h, p, n, _dev(out, name="out")))
        return out

    def backward(self, xyz, dy, dparams=None, dxyz=None):
        """Adds the parameter gradient into dparams (None: the context's gradient
        buffer); writes dL/dx of every point into dxyz ([n][3] float32) if given."""
        p, n = _points(xyz)
        dp = _dev(dparams, name="dparams") if dparams is not None else C.c_void_p()
        dx = _dev(dxyz, name="dxyz") if dxyz is not None else C.c_void_p()
        if dxyz is not None and dxyz.numel() != 3 * n:
            raise ValueError("dxyz must hold n x 3 floats")
        _check(lib().nv_backward(self._h, p, n, _dev(dy.contiguous(), name="dL_dy"), dp, dx))

    def optimizer_step(self):
        _check(lib().nv_optimizer_step(self._h))

    def train_step(self, xyz=None, target=None, n=None, vol=None, seed=0, loss_out=None):
        """One step: on a given batch (device tensors or pinned/pageable host tensors), or
        on n points sampled from `vol` (a CUDA [nz, ny, nx] tensor).  loss_out: one
        float64, on the device or in pinned host memory (valid once the step is done)."""
        lp = _loss_ptr(loss_out)
        if xyz is not None:
            for t in (xyz, target):
                if t.dtype != torch.float32 or not t.is_contiguous():
                    raise TypeError("batch tensors must be contiguous float32")
            _check(lib().nv_train_step(self._h, C.c_void_p(xyz.data_ptr()), C.c_void_p(target.data_ptr()),
                                       xyz.shape[0], None, 0, lp))
        else:
            v = volume(vol)
            _check(lib().nv_train_step(self._h, None, None, int(n), C.byref(v), int(seed), lp))

    def train_grad(self, xyz, target, n_total, loss_sum=None):
        """Forward, loss and backward of this replica's shard of a global batch of
        n_total points (nv_train_grad): the global-mean gradient is added into the
        gradient buffer, the shard's loss sum returned (one float64 on the device)."""
        if loss_sum is None:
            loss_sum = torch.zeros(1, dtype=torch.float64, device="cuda")
        p, n = _points(xyz)
        tp = _dev(target.contiguous(), name="target") if n else C.c_void_p()
        _check(lib().nv_train_grad(self._h, p, tp, n, int(n_total), _dev(loss_sum, torch.float64, "loss_sum")))
        return loss_sum

    def dp_buffers(self):
        """(gradient, flags): torch views (no copy) of the buffers a data-parallel step
        reduces across replicas -- the FP32 gradient (sum) and the int32 (overflow,
        off-domain) flags (maximum) (nv_dp_buffers)."""
        g, n, f = C.c_void_p(), C.c_int64(), C.c_void_p()
        _check(lib().nv_dp_buffers(self._h, C.byref(g), C.byref(n), C.byref(f)))
        grads = torch.as_tensor(_CudaArray(g.value, n.value), device="cuda")
        flags = torch.as_tensor(_CudaArray(f.value, 2, "<i4"), device="cuda")
        return grads, flags

    def volume_mse(self, vol, out=None):
        if out is None:
            out = torch.empty(1, dtype=torch.float64, device=vol.device)
        v = volume(vol)
        _check(lib().nv_volume_mse(self._h, C.byref(v), _dev(out, torch.float64, "out")))
        return out

    def sync(self):
        _check(lib().nv_sync(self._h))

    def profile(self, enable=True):
        _check(lib().nv_profile_enable(self._h, int(enable)))

    def profile_read(self, kclass):
        """(total device ms, launches) of one kernel class since the last read."""
        ms, n = C.c_double(), C.c_int()
        _check(lib().nv_profile_read(self._h, KCLASS[kclass] if isinstance(kclass, str) else kclass,
                                     C.byref(ms), C.byref(n)))
        return ms.value, n.value


def sample(vol, n, seed, step=0, want_xyz=True, want_target=True):
    v = volume(vol)
    xyz = torch.empty((n, 3), dtype=torch.float32, device=vol.device) if want_xyz else None
    t = torch.empty(n, dtype=torch.float32, device=vol.device) if want_target else None
    _check(lib().nv_sample(C.byref(v), int(n), int(seed), int(step),
                           C.c_void_p(xyz.data_ptr()) if xyz is not None else C.c_void_p(),
                           C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(), _stream()))
    return xyz, t


def macrocells_build(vol, cell, lut):
    v = volume(vol)
    nz, ny, nx = vol.shape
    nc = (-(-nz // cell), -(-ny // cell), -(-nx // cell))
    mm = torch.empty(nc + (2,), dtype=torch.float32, device=vol.device)
    mu = torch.empty(nc, dtype=torch.float32, device=vol.device)
    _check(lib().nv_macrocells_build(C.byref(v), int(cell), _dev(lut, name="lut"), C.c_void_p(mm.data_ptr()),
                                     C.c_void_p(mu.data_ptr()), _stream()))
    return mm, mu


class Renderer:
    """Ray-streaming buffers for images of up to max_pixels pixels (nv_renderer)."""

    def __init__(self, max_pixels, K=8, stream=None):
        h = C.c_void_p()
        s = C.c_void_p(stream) if stream is not None else _stream()
        _check(lib().nv_renderer_create(int(max_pixels), int(K), s, C.byref(h)))
        self._h = h
        self.K = K

    def close(self):
        if getattr(self, "_h", None):
            lib().nv_renderer_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def render(self, cam: dict, lut, opts: dict, net: NeuralVolume | None = None, raw=None,
               mc: tuple | None = None, out=None, rows: tuple | None = None):
        """RGBA image [H, W, 4]; net=None renders the raw volume `raw`.
        mc = (mu_max tensor, cell, raw volume shape (nz, ny, nx)) enables empty-space skipping.
        rows = (row0, n): only image rows row0 .. row0 + n - 1, as an [n, W, 4] band (nv_render_rows)."""
        c = camera(cam)
        h = c.height if rows is None else int(rows[1])
        if out is None:
            out = torch.empty((h, c.width, 4), dtype=torch.float32, device="cuda")
        elif out.numel() < h * c.width * 4:
            raise ValueError(f"out holds {out.numel()} floats, the image needs {h * c.width * 4}")
        o = render_opts(opts, self.K)
        vp = C.byref(volume(raw)) if raw is not None else None
        mp = None
        if mc is not None:
            mu, cell, shape = mc
            m = Macrocells(_dev(mu, name="mu_max").value, int(cell), int(shape[2]), int(shape[1]), int(shape[0]))
            mp = C.byref(m)
        nh = net.handle if net is not None else None
        if rows is None:
            _check(lib().nv_render(self._h, nh, vp, C.byref(c), _dev(lut, name="lut"), mp, C.byref(o),
                                   _dev(out, name="out")))
        else:
            _check(lib().nv_render_rows(self._h, nh, vp, C.byref(c), _dev(lut, name="lut"), mp, C.byref(o),
                                        int(rows[0]), int(rows[1]), _dev(out, name="out")))
        return out

    def render_pt(self, cam: dict, lut, opts: dict, mc: tuple, net: NeuralVolume | None = None, raw=None,
                  out=None):
        """One path-traced frame (nv_render_pt): RGB radiance + hit flag [H, W, 4].
        opts: density, light (unit direction to it), max_bounces (8), seed, frame."""
        c = camera(cam)
        if out is None:
            out = torch.empty((c.height, c.width, 4), dtype=torch.float32, device="cuda")
        o = PtOpts(float(opts["density"]), (C.c_float * 3)(*[float(v) for v in opts["light"]]),
                   int(opts.get("max_bounces", 8)), int(opts.get("seed", 0)), int(opts.get("frame", 0)))
        mu, cell, shape = mc
        m = Macrocells(_dev(mu, name="mu_max").value, int(cell), int(shape[2]), int(shape[1]), int(shape[0]))
        vp = C.byref(volume(raw)) if raw is not None else None
        _check(lib().nv_render_pt(self._h, net.handle if net is not None else None, vp, C.byref(c),
                                  _dev(lut, name="lut"), C.byref(m), C.byref(o), _dev(out, name="out")))
        return out

    def stats(self):
        it, sm = C.c_int(), C.c_int64()
        _check(lib().nv_render_stats(self._h, C.byref(it), C.byref(sm)))
        return it.value, sm.value


def online_macrocells(shape, cell):
    """Empty online macrocell ranges [ncz, ncy, ncx, 2] for a volume of shape (nz, ny, nx)."""
    nc = tuple(-(-int(n) // cell) for n in shape)
    mm = torch.empty(nc + (2,), dtype=torch.float32, device="cuda")
    nz, ny, nx = shape
    _check(lib().nv_macrocells_reset(_dev(mm, name="minmax"), int(nx), int(ny), int(nz), int(cell), _stream()))
    return mm


def macrocells_update(minmax, xyz, val, shape, cell):
    nz, ny, nx = shape
    _check(lib().nv_macrocells_update(_dev(xyz, name="xyz"), _dev(val, name="val"), xyz.shape[0], int(nx),
                                      int(ny), int(nz), int(cell), _dev(minmax, name="minmax"), _stream()))
    return minmax


def macrocells_mu(minmax, shape, cell, lut, out=None):
    nz, ny, nx = shape
    if out is None:
        out = torch.empty(minmax.shape[:-1], dtype=torch.float32, device="cuda")
    _check(lib().nv_macrocells_mu(_dev(minmax, name="minmax"), int(nx), int(ny), int(nz), int(cell),
                                  _dev(lut, name="lut"), _dev(out, name="mu"), _stream()))
    return out


def render_inshader(net: NeuralVolume, cam: dict, lut, opts: dict, mc: tuple | None = None, out=None,
                    samples=None):
    """In-shader ray march of `net` (nv_render_inshader): RGBA image [H, W, 4].
    mc as Renderer.render; samples (optional int64 CUDA tensor of 1) receives the
    evaluated sample count."""
    c = camera(cam)
    if out is None:
        out = torch.empty((c.height, c.width, 4), dtype=torch.float32, device="cuda")
    o = render_opts(opts, 1)
    mp = None
    if mc is not None:
        mu, cell, shape = mc
        m = Macrocells(_dev(mu, name="mu_max").value, int(cell), int(shape[2]), int(shape[1]), int(shape[0]))
        mp = C.byref(m)
    sp = _dev(samples, torch.int64, "samples") if samples is not None else None
    _check(lib().nv_render_inshader(net.handle, C.byref(c), _dev(lut, name="lut"), mp, C.byref(o),
                                    _dev(out, name="out"), sp))
    return out


PEAK_OPS_QUANTUM = 8192  # accesses per CTA of the measurement kernels


def peak_scatter(buf, ops, seed=0):
    """Issue `ops` scattered 16-byte FP32 vector reductions into buf (float32 [n16, 4], n16 a power of two)."""
    if buf.dim() != 2 or buf.shape[1] != 4:
        raise ValueError("buf must be [n16, 4] float32")
    _check(lib().nv_peak_scatter(_dev(buf, name="buf"), buf.shape[0], int(ops), int(seed), _stream()))


def peak_gather(buf, ops, sink, seed=0):
    """Issue `ops` scattered 16-byte loads from buf (any dtype, [n16 x 16 bytes]); sink: 1024 int32."""
    n16 = buf.numel() * buf.element_size() // 16
    _check(lib().nv_peak_gather(C.c_void_p(buf.data_ptr()), n16, int(ops), int(seed),
                                _dev(sink, torch.int32, "sink"), _stream()))


def image_mse(a, b, out=None):
    if a.shape != b.shape or a.shape[-1] != 4:
        raise ValueError("images must have the same [H, W, 4] shape")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=a.device)
    n = a.numel() // 4
    _check(lib().nv_image_mse(_dev(a, name="a"), _dev(b, name="b"), n, _dev(out, torch.float64, "out"), _stream()))
    return out


def mse(a, b, out=None):
    """FP64 mean squared error of two float32 CUDA tensors of the same size."""
    if a.numel() != b.numel():
        raise ValueError("mse: sizes differ")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=a.device)
    _check(lib().nv_mse_f64(_dev(a.contiguous(), name="a"), _dev(b.contiguous(), name="b"), a.numel(),
                            _dev(out, torch.float64, "out"), _stream()))
    return out


class BrickRing:
    """Out-of-core sampling ring (nv_ooc): a device ring of bricks fed from
    pinned host bricks (a CPU float32 tensor in pinned memory, kept alive here)."""

    def __init__(self, host_bricks: torch.Tensor, shape, brick, ring_slots, seed=0):
        if host_bricks.device.type != "cpu" or not host_bricks.is_pinned():
            raise ValueError("host_bricks must be a pinned CPU tensor")
        if host_bricks.dtype != torch.float32 or not host_bricks.is_contiguous():
            raise ValueError("host_bricks must be contiguous float32")
        self.host = host_bricks
        nz, ny, nx = (int(v) for v in shape)
        h = C.c_void_p()
        _check(lib().nv_ooc_create(C.c_void_p(host_bricks.data_ptr()), nx, ny, nz, int(brick), int(ring_slots),
                                   int(seed), C.byref(h)))
        self._h = h
        self.R = ring_slots

    def close(self):
        if getattr(self, "_h", None):
            lib().nv_ooc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def refresh(self, count, seed):
        _check(lib().nv_ooc_refresh(self._h, int(count), int(seed), _stream()))

    def sample(self, n, seed, step, xyz=None, target=None):
        if xyz is None:
            xyz = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        if target is None:
            target = torch.empty(n, dtype=torch.float32, device="cuda")
        _check(lib().nv_ooc_sample(self._h, int(n), int(seed), int(step), _dev(xyz, name="xyz"),
                                   _dev(target, name="target"), _stream()))
        return xyz, target

    def slots(self):
        arr = (C.c_int * self.R)()
        _check(lib().nv_ooc_slots(self._h, arr))
        return list(arr)

    def stats(self):
        b, ms = C.c_int64(), C.c_double()
        _check(lib().nv_ooc_stats(self._h, C.byref(b), C.byref(ms)))
        return b.value, ms.value


class NeuralVolumeFunction(torch.autograd.Function):
    """y = net(xyz) with the hand-written backward (A-6/A-7).

    `params` is net.parameter(): a leaf tensor viewing the network's FP32
    parameters.  The forward calls nv_infer; the backward calls nv_backward,
    which recomputes the forward (nothing is stored in between) and returns
    the parameter gradient, so torch accumulates it into params.grad, and the
    gradient in the points when xyz requires one."""

    @staticmethod
    def forward(ctx, xyz, params, net: NeuralVolume):
        ctx.net = net
        ctx.save_for_backward(xyz)
        return net.infer(xyz.detach().contiguous())

    @staticmethod
    def backward(ctx, dy):
        (xyz,) = ctx.saved_tensors
        g = torch.zeros(ctx.net.n_params, dtype=torch.float32, device=dy.device)
        gx = torch.empty_like(xyz, dtype=torch.float32) if ctx.needs_input_grad[0] else None
        ctx.net.backward(xyz.detach().contiguous(), dy.contiguous().float(), g, gx)
        return gx, g, None
