"""libdeblur Python binding: argument marshalling over the C ABI.

Every step of the Wiener + RRRL pipeline runs in the CUDA library
(`libdeblur.so`, built in-tree for sm_103a); this module only checks tensor
layouts, passes device pointers, sizes and the current CUDA stream, and turns
status codes into exceptions.  PyTorch supplies device memory and streams.
There is no CPU fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from .params import Params

__all__ = ["Params", "DeblurError", "Workspace", "workspace_bytes", "wiener", "rrl_iterate",
           "deblur", "Plan", "Batch", "deblur_batch", "rrl_backward", "DeblurFn", "rrl_iterate_noalloc", "HostBuffer", "set_schedule", "set_one_axis_min", "set_spin_limit",
           "set_rf_eval", "set_dense_min", "set_fft_tiles", "set_batch_order", "set_tma", "version", "FrameStream",
           "BatchStream", "deblur_n", "workspace_bytes_n"]


class DeblurError(RuntimeError):
    pass


def _check(code: int, what: str):
    if code != 0:
        msg = _lib.load().db_status_string(code).decode()
        raise DeblurError(f"{what}: {msg} (status {code})")


def _db_params(p: Params) -> _lib.DbParams:
    conv = {"clamp": _lib.DB_CONV_CLAMP, "periodic": _lib.DB_CONV_PERIODIC}[p.conv]
    return _lib.DbParams(float(p.K), float(p.alpha), float(p.eps_phi), float(p.eps_psi),
                         float(p.pos_floor), int(p.phi_robust), int(p.psi_tv), conv)


def _kind(kind: str) -> int:
    return _lib.DB_PSF_BOX if kind.startswith("box") else _lib.DB_PSF_GENERAL


def _db_psf(taps: torch.Tensor, kind: str) -> _lib.DbPsf:
    if not (taps.is_cuda and taps.dtype == torch.float32 and taps.dim() == 2 and taps.is_contiguous()):
        raise ValueError("taps must be a contiguous 2D float32 CUDA tensor")
    return _lib.DbPsf(taps.shape[0], taps.shape[1], _kind(kind), taps.data_ptr())


def _image(x: torch.Tensor, name: str):
    if not (x.is_cuda and x.dtype == torch.float32 and x.dim() == 2 and x.stride(1) == 1):
        raise ValueError(f"{name} must be a 2D float32 CUDA tensor with unit column stride")
    return x.shape[0], x.shape[1], x.stride(0)


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def workspace_bytes(H: int, W: int, kh: int, kw: int, params: Params) -> int:
    lib = _lib.load()
    psf = _lib.DbPsf(kh, kw, 0, None)
    p = _db_params(params)
    n = lib.db_workspace_bytes(H, W, ctypes.byref(psf), ctypes.byref(p))
    if n == 0:
        raise DeblurError("invalid size or parameters for workspace query")
    return int(n)


def workspace_bytes_n(H: int, W: int, n: int, kh: int, kw: int, params: Params) -> int:
    """Workspace of db_deblur_n for n images of H x W."""
    psf = _lib.DbPsf(kh, kw, 0, None)
    nbytes = _lib.load().db_workspace_bytes_n(H, W, n, ctypes.byref(psf), ctypes.byref(_db_params(params)))
    if nbytes == 0:
        raise DeblurError("invalid size or parameters for db_deblur_n")
    return int(nbytes)


class Workspace:
    """Caller-owned device scratch (256-byte aligned) and status word."""

    def __init__(self, nbytes: int, device=None):
        device = device or torch.device("cuda", torch.cuda.current_device())
        self.buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        off = (-self.buf.data_ptr()) % 256
        self.ptr = self.buf.data_ptr() + off
        self.nbytes = nbytes
        self.status = torch.zeros(1, dtype=torch.int32, device=device)

    @classmethod
    def for_image(cls, H, W, kh, kw, params):
        return cls(workspace_bytes(H, W, kh, kw, params))

    def reset_status(self):
        self.status.zero_()

    def raise_on_flags(self, what: str):
        flags = int(self.status.item())
        if flags:
            code = _lib.load().db_status_from_flags(flags)
            _check(code, f"{what} (device flags 0x{flags:x})")


def _ws(ws, H, W, taps, params):
    return ws if ws is not None else Workspace.for_image(H, W, taps.shape[0], taps.shape[1], params)


def wiener(f: torch.Tensor, taps: torch.Tensor, params: Params, *, kind: str = "general",
           out: torch.Tensor | None = None, ws: Workspace | None = None, check: bool = True):
    """Wiener initialisation u0 = max(Wiener(max(f, delta)), delta) (Eq. 2)."""
    H, W, ld = _image(f, "f")
    u0 = out if out is not None else torch.empty_like(f)
    if _image(u0, "out")[2] != ld or u0.shape != f.shape:
        raise ValueError("out must match f's shape and row stride")
    ws = _ws(ws, H, W, taps, params)
    if check:
        ws.reset_status()
    lib = _lib.load()
    psf, p = _db_psf(taps, kind), _db_params(params)
    _check(lib.db_wiener(f.data_ptr(), u0.data_ptr(), H, W, ld, ctypes.byref(psf), ctypes.byref(p),
                         ws.ptr, ws.nbytes, ws.status.data_ptr(), _stream()), "db_wiener")
    if check:
        ws.raise_on_flags("db_wiener")
    return u0


def rrl_iterate(f: torch.Tensor, u: torch.Tensor, taps: torch.Tensor, params: Params, iters: int, *,
                kind: str = "general", ckpt: torch.Tensor | None = None, ckpt_every: int = 0,
                ws: Workspace | None = None, check: bool = True):
    """`iters` RRRL iterations in place on u (Eq. 9-12)."""
    H, W, ld = _image(f, "f")
    if _image(u, "u")[2] != ld or u.shape != f.shape:
        raise ValueError("u must match f's shape and row stride")
    ws = _ws(ws, H, W, taps, params)
    if check:
        ws.reset_status()
    ck = 0
    if ckpt is not None:
        nck = (iters - 1) // ckpt_every + 1 if iters > 0 else 0
        if not (ckpt.is_cuda and ckpt.dtype == torch.float32 and ckpt.is_contiguous()
                and ckpt.numel() >= nck * H * W):
            raise ValueError("ckpt must be a contiguous float32 CUDA tensor of (iters-1)//every+1 images")
        ck = ckpt.data_ptr()
    lib = _lib.load()
    psf, p = _db_psf(taps, kind), _db_params(params)
    _check(lib.db_rrl_iterate(f.data_ptr(), u.data_ptr(), H, W, ld, ctypes.byref(psf), ctypes.byref(p),
                              int(iters), ck, int(ckpt_every), ws.ptr, ws.nbytes, ws.status.data_ptr(),
                              _stream()), "db_rrl_iterate")
    if check:
        ws.raise_on_flags("db_rrl_iterate")
    return u


def deblur(f: torch.Tensor, taps: torch.Tensor, params: Params, iters: int, *, kind: str = "general",
           out: torch.Tensor | None = None, ws: Workspace | None = None, check: bool = True):
    """Whole WR3L pipeline: Wiener, floor, `iters` RRRL iterations (Sec. 3.2)."""
    H, W, ld = _image(f, "f")
    u = out if out is not None else torch.empty_like(f)
    ws = _ws(ws, H, W, taps, params)
    if check:
        ws.reset_status()
    lib = _lib.load()
    psf, p = _db_psf(taps, kind), _db_params(params)
    _check(lib.db_deblur(f.data_ptr(), u.data_ptr(), H, W, ld, ctypes.byref(psf), ctypes.byref(p),
                         int(iters), ws.ptr, ws.nbytes, ws.status.data_ptr(), _stream()), "db_deblur")
    if check:
        ws.raise_on_flags("db_deblur")
    return u


def deblur_n(f: torch.Tensor, taps: torch.Tensor, params: Params, iters: int, *, kind: str = "general",
             out: torch.Tensor | None = None, ckpt: torch.Tensor | None = None, ckpt_every: int = 0,
             ws: Workspace | None = None, check: bool = True):
    """WR3L on a stack f (N, H, W) of equally sized images sharing taps and
    parameters (db_deblur_n): the iterations run as launches over all images
    at once.  ckpt (N, nck, H, W), if given, receives every image's iterate
    at iterations 0, ckpt_every, 2*ckpt_every, ... (nck = (iters-1)//ckpt_every+1)."""
    if f.dim() != 3 or not f.is_cuda or f.dtype != torch.float32 or f.stride(2) != 1:
        raise ValueError("f must be a (N, H, W) float32 CUDA tensor with unit column stride")
    N, H, W = f.shape
    ld, zs = f.stride(1), f.stride(0)
    u = out if out is not None else torch.empty_strided(f.shape, f.stride(), dtype=f.dtype, device=f.device)
    if u.shape != f.shape or u.stride() != f.stride():
        raise ValueError("out must match f's shape and strides")
    ck, every = 0, 0
    if ckpt is not None:
        if ckpt_every < 1:
            raise ValueError("ckpt_every must be >= 1")
        nck = (iters - 1) // ckpt_every + 1 if iters > 0 else 1
        if not (ckpt.is_cuda and ckpt.dtype == torch.float32 and ckpt.is_contiguous()
                and ckpt.numel() >= N * nck * H * W):
            raise ValueError("ckpt must be a contiguous float32 CUDA tensor of N x nck images")
        ck, every = ckpt.data_ptr(), int(ckpt_every)
    lib = _lib.load()
    psf, p = _db_psf(taps, kind), _db_params(params)
    if ws is None:
        ws = Workspace(workspace_bytes_n(H, W, N, taps.shape[0], taps.shape[1], params))
    elif check:
        ws.reset_status()
    _check(lib.db_deblur_n(f.data_ptr(), u.data_ptr(), H, W, ld, N, zs, ctypes.byref(psf), ctypes.byref(p),
                           int(iters), ck, every, ws.ptr, ws.nbytes, ws.status.data_ptr(), _stream()), "db_deblur_n")
    if check:
        ws.raise_on_flags("db_deblur_n")
    return u


class Plan:
    """Prepared single-image pipeline (db_plan_create): transform tables, PSF
    spectrum and tap groups computed once for an image size, PSF and
    parameters; `run(f, out)` applies Wiener + `iters` RRRL (capturable).
    The result equals deblur()'s bit for bit."""

    def __init__(self, H: int, W: int, taps: torch.Tensor, params: Params, iters: int, *,
                 kind: str = "general", ld: int | None = None):
        ld = W if ld is None else ld
        self.taps = taps
        self.ws = Workspace.for_image(H, W, taps.shape[0], taps.shape[1], params)
        self.ws.reset_status()
        lib = _lib.load()
        psf, p = _db_psf(taps, kind), _db_params(params)
        h = ctypes.c_void_p()
        _check(lib.db_plan_create(H, W, ld, ctypes.byref(psf), ctypes.byref(p), int(iters), self.ws.ptr,
                                  self.ws.nbytes, self.ws.status.data_ptr(), _stream(), ctypes.byref(h)),
               "db_plan_create")
        self._h = h
        self.shape, self.ld = (H, W), ld

    def run(self, f: torch.Tensor, out: torch.Tensor | None = None, check: bool = True):
        H, W, ld = _image(f, "f")
        if (H, W) != self.shape or ld != self.ld:
            raise ValueError("image shape or row stride differs from the plan's")
        u = out if out is not None else torch.empty_like(f)
        if check:
            self.ws.reset_status()
        _check(_lib.load().db_plan_run(self._h, f.data_ptr(), u.data_ptr(), self.ws.status.data_ptr(), _stream()),
               "db_plan_run")
        if check:
            self.ws.raise_on_flags("db_plan_run")
        return u

    def autotune(self, f: torch.Tensor, reps: int = 3):
        """Pick this plan's schedule by timing every form on f (db_plan_autotune;
        synchronises the current stream).  Returns (schedule, one_axis_form):
        schedule one of "split", "flow", "fused" (None for a periodic plan),
        form "groups" (direct sums), "windows", "fft" or None."""
        u = torch.empty_like(f)
        cs, ca = ctypes.c_int(-1), ctypes.c_int(-1)
        self.ws.reset_status()
        _check(_lib.load().db_plan_autotune(self._h, f.data_ptr(), u.data_ptr(), int(reps),
                                            self.ws.status.data_ptr(), _stream(), ctypes.byref(cs),
                                            ctypes.byref(ca)), "db_plan_autotune")
        self.ws.raise_on_flags("db_plan_autotune")
        names = {_lib.SCHED_SPLIT: "split", _lib.SCHED_FLOW: "flow", _lib.SCHED_FUSED: "fused",
                 _lib.SCHED_CLUSTER: "cluster"}
        return names.get(cs.value), {0: "groups", 2: "windows", 3: "fft"}.get(ca.value)

    def run_host(self, f_host, u_host, check: bool = True, sync: bool = True):
        """The pipeline on an image in host memory (db_plan_run_host): the
        copy in, the run and the copy out are enqueued on the current stream,
        which is synchronised before returning (unless sync=False; then
        check must be False too).  f_host and u_host are H x W float32 host
        buffers: HostBuffer (page-locked, the fast path) or contiguous CPU
        tensors."""
        if check and not sync:
            raise ValueError("check=True needs sync=True")
        H, W = self.shape
        fp, up = _host_ptr(f_host, (H, W), "f_host"), _host_ptr(u_host, (H, W), "u_host")
        if getattr(self, "_dev", None) is None:
            self._dev = (torch.empty(H, self.ld, device="cuda"), torch.empty(H, self.ld, device="cuda"))
        fd, ud = self._dev
        if check:
            self.ws.reset_status()
        _check(_lib.load().db_plan_run_host(self._h, fp, up, fd.data_ptr(), ud.data_ptr(),
                                            self.ws.status.data_ptr(), _stream()), "db_plan_run_host")
        if sync:
            torch.cuda.current_stream().synchronize()
        if check:
            self.ws.raise_on_flags("db_plan_run_host")
        return u_host

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().db_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostBuffer:
    """Page-locked host memory from db_host_alloc, viewed as a float32 CPU
    tensor (`.tensor`, which shares the memory: keep the HostBuffer alive
    while using it).  Copies from and to it run at the link's full rate."""

    def __init__(self, shape):
        self.shape = tuple(int(x) for x in shape)
        n = 1
        for x in self.shape:
            n *= x
        ptr = ctypes.c_void_p()
        _check(_lib.load().db_host_alloc(max(n, 1) * 4, ctypes.byref(ptr)), "db_host_alloc")
        self._ptr = ptr
        arr = np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctypes.c_float)), shape=self.shape)
        self.tensor = torch.from_numpy(arr)

    @property
    def ptr(self) -> int:
        return self._ptr.value

    def copy_from(self, array) -> "HostBuffer":
        """Fill from a host array of the same shape with one single-threaded
        copy.  (Rows written by many host threads can sit dirty in the caches
        of several cores; the device's reads of them then ran five times
        slower on B300 hosts than after a single-threaded copy.)"""
        a = np.ascontiguousarray(np.asarray(array, dtype=np.float32))
        if a.shape != self.shape:
            raise ValueError(f"shape {a.shape} != {self.shape}")
        ctypes.memmove(self.ptr, a.ctypes.data, a.nbytes)
        return self

    def close(self):
        if getattr(self, "_ptr", None) is not None and self._ptr.value:
            self.tensor = None
            _lib.load().db_host_free(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _host_ptr(buf, shape, what: str) -> int:
    if isinstance(buf, HostBuffer):
        if buf.shape != tuple(shape):
            raise ValueError(f"{what}: shape {buf.shape} != {tuple(shape)}")
        return buf.ptr
    if not isinstance(buf, torch.Tensor) or buf.device.type != "cpu" or buf.dtype != torch.float32 \
            or not buf.is_contiguous() or tuple(buf.shape) != tuple(shape):
        raise ValueError(f"{what}: expected a contiguous float32 CPU tensor of shape {tuple(shape)} or a HostBuffer")
    return buf.data_ptr()


class Batch:
    """A planned batch of images (uneven sizes, own PSF and parameters each):
    `run()` deblurs all of them (Wiener + `iters` RRRL) with five batched
    Wiener launches and one persistent RRRL launch; it enqueues launches and
    memsets only, so it can be captured in a CUDA graph.  The plan refers to
    the given tensors: keep them alive; their values may change between runs."""

    def __init__(self, fs, taps, params, iters, *, kinds=None, outs=None):
        n = len(fs)
        if not (len(taps) == n and (not isinstance(params, (list, tuple)) or len(params) == n)):
            raise ValueError("fs, taps and params must have the same length")
        params = list(params) if isinstance(params, (list, tuple)) else [params] * n
        kinds = list(kinds) if kinds is not None else ["general"] * n
        self.fs = list(fs)
        self.taps = list(taps)
        self.us = list(outs) if outs is not None else [torch.empty_like(f) for f in self.fs]
        descs = (_lib.DbImageDesc * n)()
        for k in range(n):
            H, W, ld = _image(self.fs[k], "f")
            if _image(self.us[k], "u")[2] != ld or self.us[k].shape != self.fs[k].shape:
                raise ValueError("outputs must match the inputs' shapes and row strides")
            descs[k] = _lib.DbImageDesc(self.fs[k].data_ptr(), self.us[k].data_ptr(), H, W, ld,
                                        _db_psf(self.taps[k], kinds[k]), _db_params(params[k]))
        self._descs = descs
        lib = _lib.load()
        nbytes = lib.db_batch_workspace_bytes(descs, n, int(iters))
        if nbytes == 0:
            raise DeblurError("invalid batch descriptors")
        self.ws = Workspace(nbytes)
        self.ws.reset_status()
        handle = ctypes.c_void_p()
        _check(lib.db_batch_create(descs, n, int(iters), self.ws.ptr, self.ws.nbytes,
                                   self.ws.status.data_ptr(), _stream(), ctypes.byref(handle)),
               "db_batch_create")
        self._h = handle
        self.iters = iters

    def run(self, check: bool = True):
        if check:
            self.ws.reset_status()
        _check(_lib.load().db_batch_run(self._h, self.ws.status.data_ptr(), _stream()), "db_batch_run")
        if check:
            self.ws.raise_on_flags("db_batch_run")
        return self.us

    def autotune(self, reps: int = 3):
        """Choose the tile forms by timing whole runs (db_batch_autotune):
        register windows or tap groups for non-box one-axis PSFs, the dense
        sums on or off for dense-eligible 2D PSFs, and the FFT-tile threshold
        on kh * kw for 2D PSFs.  Overwrites the outputs and synchronises the
        current stream.  Returns {"fft": t, "dense": bool, "windows": w} with t
        the threshold (0: no FFT tiles; set_fft_tiles(t or 2305) reproduces
        it), w = "rule" (the size rule of set_one_axis_min(0)), "all"
        (register windows) or "none" (tap groups)."""
        d, w, ft = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self.ws.reset_status()
        _check(_lib.load().db_batch_autotune(self._h, int(reps), self.ws.status.data_ptr(), _stream(),
                                             ctypes.byref(d), ctypes.byref(w), ctypes.byref(ft)),
               "db_batch_autotune")
        self.ws.raise_on_flags("db_batch_autotune")
        return {"fft": int(ft.value), "dense": bool(d.value),
                "windows": {0: "none", 1: "all", 2: "rule"}[w.value]}

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().db_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def deblur_batch(fs, taps, params, iters, *, kinds=None, outs=None, check: bool = True):
    """Deblur a list of images in one batched run; returns the outputs."""
    b = Batch(fs, taps, params, iters, kinds=kinds, outs=outs)
    try:
        return b.run(check=check)
    finally:
        b.close()


def rrl_backward(f, ckpt, grad_u, taps, params, iters, ckpt_every, grad_taps, grad_alpha, grad_K, *,
                 grad_f=None, ws=None, check: bool = True):
    """Reverse mode of Wiener + `iters` RRRL (db_rrl_backward) for one image
    (H, W) or a batch (N, H, W) sharing taps and parameters; ckpt holds each
    image's checkpoints ((N,) nck, H, W).  grad_taps/grad_alpha/grad_K are
    float64 CUDA tensors accumulated in place."""
    batched = f.dim() == 3
    fb = f if batched else f.unsqueeze(0)
    N, H, W = fb.shape
    if not (fb.is_cuda and fb.dtype == torch.float32 and fb.is_contiguous()):
        raise ValueError("f must be a contiguous float32 CUDA tensor")
    gu = grad_u.reshape(N, H, W)
    if not gu.is_contiguous() or not ckpt.is_contiguous():
        raise ValueError("grad_u and ckpt must be contiguous")
    gf = grad_f if grad_f is not None else torch.empty_like(f)
    lib = _lib.load()
    psf, p = _db_psf(taps, "general"), _db_params(params)
    if ws is None:
        n = lib.db_backward_workspace_bytes(H, W, N, ctypes.byref(psf), int(ckpt_every))
        if n == 0:
            raise DeblurError("invalid arguments for the backward workspace query")
        ws = Workspace(n)
    if check:
        ws.reset_status()
    for t in (grad_taps, grad_alpha, grad_K):
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError("parameter gradients must be contiguous float64 CUDA tensors")
    _check(lib.db_rrl_backward(fb.data_ptr(), ckpt.data_ptr(), gu.data_ptr(), H, W, W, N, ctypes.byref(psf),
                               ctypes.byref(p), int(iters), int(ckpt_every), gf.data_ptr(), grad_taps.data_ptr(),
                               grad_alpha.data_ptr(), grad_K.data_ptr(), ws.ptr, ws.nbytes,
                               ws.status.data_ptr(), _stream()), "db_rrl_backward")
    if check:
        ws.raise_on_flags("db_rrl_backward")
    return gf


class DeblurFn(torch.autograd.Function):
    """Differentiable WR3L for a batch f (N, H, W) with learnable one-row taps
    (1, kw), alpha and K (0-dim tensors).  Forward: db_wiener + db_rrl_iterate
    with checkpoints every `ckpt_every` iterations; backward: db_rrl_backward
    per image (gradients for f, taps, alpha and K)."""

    @staticmethod
    def forward(ctx, f, taps, alpha, K, params, iters, ckpt_every):
        import dataclasses
        p = dataclasses.replace(params, alpha=float(alpha), K=float(K))
        N, H, W = f.shape
        taps_c = taps.detach().float().contiguous()
        nck = (iters - 1) // ckpt_every + 1 if iters > 0 else 1
        ckpts = torch.empty(N, nck, H, W, dtype=torch.float32, device=f.device)
        f = f.contiguous()
        out = deblur_n(f, taps_c, p, iters, ckpt=ckpts, ckpt_every=ckpt_every, check=False)
        ctx.save_for_backward(f, taps_c, ckpts)
        ctx.p, ctx.iters, ctx.every = p, iters, ckpt_every
        return out

    @staticmethod
    def backward(ctx, grad_u):
        f, taps_c, ckpts = ctx.saved_tensors
        N, H, W = f.shape
        grad_u = grad_u.contiguous().float()
        gt = torch.zeros(taps_c.numel(), dtype=torch.float64, device=f.device)
        ga = torch.zeros(1, dtype=torch.float64, device=f.device)
        gk = torch.zeros(1, dtype=torch.float64, device=f.device)
        gf = torch.empty_like(f)
        rrl_backward(f.contiguous(), ckpts, grad_u, taps_c, ctx.p, ctx.iters, ctx.every, gt, ga, gk, grad_f=gf)
        return gf, gt.reshape(taps_c.shape).float(), ga[0].float(), gk[0].float(), None, None, None


def set_spin_limit(cycles: int):
    """Clock-cycle budget of the library's bounded device waits."""
    _check(_lib.load().db_set_spin_limit(int(cycles)), "db_set_spin_limit")


def set_batch_order(name: str):
    """Tile order of batches created after the call: "barrier" (default:
    phases separated by grid barriers) or "dependency" (each tile waits only
    for its own image's previous phase).  Both give the same bits."""
    code = {"dependency": 0, "barrier": 1}[name]
    _check(_lib.load().db_set_batch_order(code), "db_set_batch_order")


def set_tma(on: bool):
    """Stage the FFT tiles' q-phase windows by TMA tensor copies (True, the
    default) or by element-wise clamped loads (False).  Both give the same
    bits."""
    _check(_lib.load().db_set_tma(1 if on else 0), "db_set_tma")


def rrl_iterate_noalloc(f: torch.Tensor, u: torch.Tensor, taps: torch.Tensor, params: Params,
                        iters: int, *, kind: str = "general", status: torch.Tensor | None = None):
    """`iters` RRRL iterations in place on u without any device allocation:
    for callers that cannot allocate at run time (a fixed-latency frame loop,
    a plugin inside a framework that owns the GPU memory).  Scratch comes from
    a fixed array inside the library (shared by all calls on a device: do not
    overlap calls on the GPU).  `status`, if given, is a device int32 word the
    library ORs error flags into; the caller zeroes and reads it."""
    H, W, ld = _image(f, "f")
    if _image(u, "u")[2] != ld or u.shape != f.shape:
        raise ValueError("u must match f's shape and row stride")
    lib = _lib.load()
    psf, p = _db_psf(taps, kind), _db_params(params)
    st = status.data_ptr() if status is not None else None
    _check(lib.db_rrl_iterate_noalloc(f.data_ptr(), u.data_ptr(), H, W, ld, ctypes.byref(psf),
                                      ctypes.byref(p), int(iters), st, _stream()),
           "db_rrl_iterate_noalloc")
    return u


def set_schedule(name: str):
    """Kernel schedule of the spatial iteration: "auto", "fused", "split", "flow" or
    "cluster" (one-row PSFs on small images: the image resident in one cluster)."""
    code = {"auto": _lib.SCHED_AUTO, "fused": _lib.SCHED_FUSED, "split": _lib.SCHED_SPLIT,
            "flow": _lib.SCHED_FLOW, "cluster": _lib.SCHED_CLUSTER}[name]
    _check(_lib.load().db_set_schedule(code), "db_set_schedule")


def set_one_axis_min(min_len: int = 0):
    """Shortest non-box one-axis PSF summed with register windows in the split
    and flow schedules (shorter ones use tap groups); 256 = never, 0 = the
    default (rows from 16 taps, columns from 32).  Process-wide."""
    _check(_lib.load().db_set_one_axis_min(int(min_len)), "db_set_one_axis_min")


def set_dense_min(percent: int = 0):
    """Smallest share (percent) of non-zero taps for which an eligible 2D PSF
    (odd sides 3..25) is summed densely; 101 = never, 0 = the default (50).
    Process-wide; applies to taps prepared after the call."""
    _check(_lib.load().db_set_dense_min(int(percent)), "db_set_dense_min")


def set_fft_tiles(min_taps: int = 0):
    """Smallest kh * kw for which a 2D PSF (sides 2..48) runs the split
    schedule's blur and correlations as 64 x 64 FFT tiles; 2305 = never,
    0 = the default (225).  Process-wide; applies to later runs and
    batches."""
    _check(_lib.load().db_set_fft_tiles(int(min_taps)), "db_set_fft_tiles")


def set_rf_eval(name: str):
    """Evaluation of r_f in the robust weight, process-wide: "log1p" (default)
    or "lut" (the lookup table of Sec. 4.1)."""
    code = {"log1p": _lib.RF_LOG1P, "lut": _lib.RF_LUT}[name]
    _check(_lib.load().db_set_rf_eval(code), "db_set_rf_eval")


def version() -> str:
    return _lib.load().db_version().decode()


from .stream import FrameStream  # noqa: E402  (uses Plan)
from .batch_stream import BatchStream  # noqa: E402  (uses Batch)
