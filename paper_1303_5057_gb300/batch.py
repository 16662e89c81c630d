"""Batched tracing: many (a, i) images of uneven size in one persistent launch.

All images share one state buffer (image after image); one ``gray_setup``
writes every initial state, one ``gray_plan`` orders every ray of every image
longest-first (the two fused in ``gray_setup_plan`` when planning), one
``gray_trace`` traces them all, and one ``gray_shadow``
reduces each image to its captured area, equivalent radius and centroid (the
quantities behind the paper's photon-ring study, Sec. 4).  The trace step can
be captured once in a CUDA graph and replayed for further batches of the same
shape (set-up and planning copy host tables, so they stay outside the graph).
"""
from __future__ import annotations

import time

import numpy as np

from . import gray


class ShadowSweep:
    """One batch of images traced together.

    images: objects with a, M, r_obs, incl, nx, ny, alpha0/1, beta0/1 (see
    ``inputs.Image``).  opt: ``gray.Options``.  plan: order the queue
    longest-first with ``gray_plan`` (probe_stride, probe_budget)."""

    def __init__(self, images, opt: gray.Options, plan: bool = True, probe_stride: int = 6,
                 probe_budget: int = 400, device="cuda"):
        import torch
        self.images = list(images)
        self.opt = opt
        self.plan = plan
        self.probe_stride = probe_stride
        self.probe_budget = probe_budget
        self.n = sum(int(im.nx) * int(im.ny) for im in self.images)
        self.tracer = gray.Tracer(opt, self.n, device=device)
        self.order = torch.empty(max(1, self.n), dtype=torch.int32, device=device)
        self.shadow_buf = torch.empty(gray.SHADOW_DTYPE.itemsize * len(self.images), dtype=torch.uint8,
                                      device=device)
        self.graph = None

    def close(self):
        self.tracer.close()

    # -- the three phases -------------------------------------------------
    def setup(self, stream=None):
        if self.plan:
            return self.tracer.setup_plan(self.images, probe_stride=self.probe_stride,
                                          probe_budget=self.probe_budget, order=self.order, stream=stream)
        self.tracer.setup(self.images, stream=stream)
        return None

    def trace(self, order=None, stream=None):
        return self.tracer.trace(wait=False, order=order, stream=stream)

    def shadows(self, stream=None):
        gray.gray_shadow(self.tracer.ctx, self.tracer.state, self.n, self.images, out=self.shadow_buf,
                         stream=stream)
        return self.shadow_buf

    # -- one full batch -----------------------------------------------------
    def run(self):
        """Set up, plan, trace and reduce one batch; returns (shadow records,
        stats of the trace (steps, euler, fp64 steps, active), elapsed ms)."""
        import torch
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        order = self.setup()
        if self.graph is not None:
            self.graph.replay()
        else:
            self.trace(order)
        sh = self.shadows()
        torch.cuda.synchronize()
        ms = 1000.0 * (time.perf_counter() - t0)
        return gray.as_numpy(sh, gray.SHADOW_DTYPE), ms

    def capture(self):
        """Capture the trace step (epoch bump, queue reset, single pass, zone
        pass) in a CUDA graph; later ``run`` calls replay it."""
        import torch
        order = self.setup()
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.trace(order, stream=s)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = g
        return g

    def stats(self):
        """Per-ray records of the last batch (n x 17)."""
        return self.tracer.records()


def total_steps(records: np.ndarray) -> int:
    return int(records[:, 1].sum())
