"""Streaming form of the pipeline: a sequence of frames of one size, PSF and
parameter set, with the host<->device transfers overlapped with the
computation (the paper measures the transfers separately, Sec. 5.3, and
stresses that precomputed data must be reused across images).

One plan (tables, PSF spectrum, tap groups: set up once) serves all frames.
Its run is captured once per device slot in a CUDA graph.  Frames cycle
through `depth` device slots: while the compute stream deblurs frame k, an
upload stream copies frame k+1 in from pinned host memory and a download
stream copies frame k-1's result out.  Events order the three queues:
    upload(k) -> compute(k) -> download(k),
    compute(k - depth) done before upload(k) overwrites its input slot,
    download(k - depth) done before compute(k) overwrites its output slot.
"""
from __future__ import annotations

import torch

from . import Plan
from .params import Params


class FrameStream:
    def __init__(self, H: int, W: int, taps: torch.Tensor, params: Params, iters: int, *,
                 kind: str = "general", depth: int = 2, device=None):
        if depth < 2:
            raise ValueError("depth must be >= 2 for transfers to overlap")
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.shape = (H, W)
        self.depth = depth
        self.compute = torch.cuda.Stream(device=self.device)
        self.h2d = torch.cuda.Stream(device=self.device)
        self.d2h = torch.cuda.Stream(device=self.device)
        self.f = [torch.empty(H, W, device=self.device) for _ in range(depth)]
        self.u = [torch.empty(H, W, device=self.device) for _ in range(depth)]
        with torch.cuda.stream(self.compute):
            self.plan = Plan(H, W, taps, params, iters, kind=kind)
            for t in self.f:
                t.fill_(max(1.0, params.pos_floor))
            for s in range(depth):  # first run outside capture: module loading, attributes
                self.plan.run(self.f[s], self.u[s])
            self.graphs = []
            for s in range(depth):
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=self.compute):
                    self.plan.run(self.f[s], self.u[s], check=False)
                self.graphs.append(g)
        self.compute.synchronize()
        self._ev = lambda: torch.cuda.Event()  # noqa: E731

    def run(self, frames, outs=None):
        """Deblur host frames (pinned float32 H x W tensors) into host outputs
        (pinned; allocated if not given).  Returns the outputs once all are
        on the host."""
        n = len(frames)
        if outs is None:
            outs = [torch.empty(self.shape, dtype=torch.float32).pin_memory() for _ in range(n)]
        up = [None] * n
        done = [None] * n
        down = [None] * n
        with torch.cuda.stream(self.compute):
            self.plan.ws.reset_status()
        for k in range(n):
            s = k % self.depth
            with torch.cuda.stream(self.h2d):
                if k >= self.depth:
                    self.h2d.wait_event(done[k - self.depth])  # input slot free
                self.f[s].copy_(frames[k], non_blocking=True)
                up[k] = self._ev()
                up[k].record(self.h2d)
            with torch.cuda.stream(self.compute):
                self.compute.wait_event(up[k])
                if k >= self.depth:
                    self.compute.wait_event(down[k - self.depth])  # output slot free
                self.graphs[s].replay()
                done[k] = self._ev()
                done[k].record(self.compute)
            with torch.cuda.stream(self.d2h):
                self.d2h.wait_event(done[k])
                outs[k].copy_(self.u[s], non_blocking=True)
                down[k] = self._ev()
                down[k].record(self.d2h)
        self.d2h.synchronize()
        self.compute.synchronize()
        self.plan.ws.raise_on_flags("streamed frames")
        return outs

    def close(self):
        self.plan.close()
