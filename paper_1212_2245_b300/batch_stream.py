"""A batch of host images deblurred with the transfers overlapped.

The images are split into `parts` planned sub-batches of about equal work
(longest-processing-time assignment on pixels x iterations).  An upload
stream copies every sub-batch's images in from page-locked host memory; the
compute stream replays sub-batch k's captured run as soon as its copies have
landed; a download stream copies sub-batch k's results out as soon as its run
has finished.  So the copies of later sub-batches overlap the runs of earlier
ones, and the results of earlier ones go out while later ones run.  Events
order the three queues:
    upload(k) -> compute(k) -> download(k)
and, across calls,
    compute(k) of the previous call before upload(k) overwrites its inputs,
    download(k) of the previous call before compute(k) overwrites its outputs.
Each sub-batch is an ordinary Batch, whose images equal single-image runs bit
for bit, so the results do not depend on `parts`.
"""
from __future__ import annotations

import torch

from . import Batch, shard


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
        self.fs = [torch.empty(s, device=self.device) for s in self.shapes]
        self.us = [torch.empty(s, device=self.device) for s in self.shapes]
        costs = shard.image_costs(self.shapes, iters)
        self.parts = [p for p in shard.lpt_partition(costs, min(parts, n)) if p]
        self.compute = torch.cuda.Stream(device=self.device)
        self.up = torch.cuda.Stream(device=self.device)
        self.down = torch.cuda.Stream(device=self.device)
        self.batches, self.graphs = [], []
        with torch.cuda.stream(self.compute):
            for idx in self.parts:
                for i in idx:  # any positive image for the first run
                    self.fs[i].fill_(max(1.0, float(params[i].pos_floor)))
                b = Batch([self.fs[i] for i in idx], [taps[i] for i in idx], [params[i] for i in idx], iters,
                          kinds=[kinds[i] for i in idx], outs=[self.us[i] for i in idx])
                b.run()  # first run outside capture: module loading, attributes
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=self.compute):
                    b.run(check=False)
                self.batches.append(b)
                self.graphs.append(g)
        self.compute.synchronize()
        self._done = [None] * len(self.parts)   # compute finished (previous call)
        self._down = [None] * len(self.parts)   # download finished (previous call)

    def run(self, f_host, u_host, sync: bool = True):
        """Deblur host images f_host[i] (page-locked float32, shape shapes[i])
        into u_host[i].  With sync=False the call returns once everything is
        enqueued; the caller synchronises the download stream (`self.down`)."""
        if len(f_host) != len(self.shapes) or len(u_host) != len(self.shapes):
            raise ValueError("one host input and one host output per image")
        for b in self.batches:
            with torch.cuda.stream(self.compute):
                b.ws.reset_status()
        ups = []
        for k, idx in enumerate(self.parts):
            with torch.cuda.stream(self.up):
                if self._done[k] is not None:
                    self.up.wait_event(self._done[k])  # the previous run no longer reads these inputs
                for i in idx:
                    self.fs[i].copy_(f_host[i], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(self.up)
                ups.append(ev)
        for k, idx in enumerate(self.parts):
            with torch.cuda.stream(self.compute):
                self.compute.wait_event(ups[k])
                if self._down[k] is not None:
                    self.compute.wait_event(self._down[k])  # the previous download has read the outputs
                self.graphs[k].replay()
                done = torch.cuda.Event()
                done.record(self.compute)
                self._done[k] = done
            with torch.cuda.stream(self.down):
                self.down.wait_event(done)
                for i in idx:
                    u_host[i].copy_(self.us[i], non_blocking=True)
                dn = torch.cuda.Event()
                dn.record(self.down)
                self._down[k] = dn
        if sync:
            self.down.synchronize()
            self.compute.synchronize()
            for b in self.batches:
                b.ws.raise_on_flags("streamed batch")
        return u_host

    def close(self):
        for b in self.batches:
            b.close()
        self.batches = []
