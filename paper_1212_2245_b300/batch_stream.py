"""A batch of host images deblurred with the transfers overlapped.

A thin binding of the library's streamed batch (db_batch_stream_*): the
images are split into `parts` sub-batches whose pixel counts ramp up from
the first and down to the last (shares 1, 4, 16, ..., 16, 4, 1); for
each sub-batch the library copies its host images in on an upload stream,
runs it on the caller's stream once they have landed, and copies its
results out on a download stream, so the transfers of the other sub-batches
overlap each run.  Synchronising the caller's stream makes the host results
valid.  Each sub-batch is an ordinary planned batch, whose images equal
single-image runs bit for bit, so the results do not depend on `parts`.
"""
from __future__ import annotations

import ctypes

import torch

from . import DeblurError, Workspace, _check, _db_params, _db_psf, _lib, _stream


class BatchStream:
    def __init__(self, shapes, taps, params, iters: int, *, kinds=None, parts: int = 4, device=None):
        n = len(shapes)
        if len(taps) != n:
            raise ValueError("shapes and taps must have the same length")
        if parts < 1:
            raise ValueError("parts must be >= 1")
        params = list(params) if isinstance(params, (list, tuple)) else [params] * n
        kinds = list(kinds) if kinds is not None else ["general"] * n
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.shapes = [tuple(int(x) for x in s) for s in shapes]
        # device staging buffers of the library's copies
        self.fs = [torch.empty(s, device=self.device) for s in self.shapes]
        self.us = [torch.empty(s, device=self.device) for s in self.shapes]
        self.taps = list(taps)
        descs = (_lib.DbImageDesc * n)()
        for k, (H, W) in enumerate(self.shapes):
            descs[k] = _lib.DbImageDesc(self.fs[k].data_ptr(), self.us[k].data_ptr(), H, W, W,
                                        _db_psf(self.taps[k], kinds[k]), _db_params(params[k]))
        self._descs = descs
        lib = _lib.load()
        nbytes = lib.db_batch_stream_workspace_bytes(descs, n, int(iters), int(parts))
        if nbytes == 0:
            raise DeblurError("invalid batch descriptors")
        self.ws = Workspace(nbytes, self.device)
        self.ws.reset_status()
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib.db_batch_stream_create(descs, n, int(iters), int(parts), self.ws.ptr, self.ws.nbytes,
                                              self.ws.status.data_ptr(), _stream(), ctypes.byref(h)),
                   "db_batch_stream_create")
        self._h = h
        self.parts = int(lib.db_batch_stream_parts(h))
        torch.cuda.current_stream(self.device).synchronize()

    def run(self, f_host, u_host, sync: bool = True):
        """Deblur host images f_host[i] (float32, shape shapes[i], contiguous;
        page-locked for overlapped copies) into u_host[i], on the current
        stream.  With sync=False the call returns once everything is enqueued;
        the results are valid after the current stream has been synchronised."""
        n = len(self.shapes)
        if len(f_host) != n or len(u_host) != n:
            raise ValueError("one host input and one host output per image")
        fp = (ctypes.c_void_p * n)()
        up = (ctypes.c_void_p * n)()
        for i, (a, b) in enumerate(zip(f_host, u_host)):
            for t, what in ((a, "f_host"), (b, "u_host")):
                if t.device.type != "cpu" or t.dtype != torch.float32 or not t.is_contiguous() or \
                        tuple(t.shape) != self.shapes[i]:
                    raise ValueError(f"{what}[{i}] must be a contiguous float32 host tensor of shape {self.shapes[i]}")
            fp[i], up[i] = a.data_ptr(), b.data_ptr()
        if sync:
            self.ws.reset_status()
        _check(_lib.load().db_batch_stream_run_host(self._h, fp, up, self.ws.status.data_ptr(), _stream()),
               "db_batch_stream_run_host")
        if sync:
            torch.cuda.current_stream(self.device).synchronize()
            self.ws.raise_on_flags("streamed batch")
        return u_host

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().db_batch_stream_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
