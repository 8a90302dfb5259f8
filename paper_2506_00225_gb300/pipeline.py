"""Streaming mapping step: targets arrive from host memory every step.

``MappingStream`` captures the fused mapping step (project, bin/sort,
forward render fused with the mean-L1 loss of Sec. 3.1 Eq. 2's colour and
depth terms plus the semantic L1 term, and the adjoint to every Gaussian
parameter) as one CUDA graph per device input slot.  ``step`` copies the
next frame's targets from pinned host memory into the free slot on a copy
stream, so the host-to-device transfer of frame i + 1 runs while the graph of
frame i computes; each step's loss is read back to pinned host memory.

The arithmetic is that of ``raster.render_l1`` followed by its backward: the
graphs only fix the launch sequence, the buffers and the streams.
"""
from __future__ import annotations

import torch

from . import raster


class MappingStream:
    """Double-buffered, graph-captured mapping steps for one camera.

    Parameters: a ``Rasterizer`` (owns the workspace; sized by a first
    ``forward`` with ``check=True`` before capture), the ``Gaussians`` (their
    ids and class count), the camera, the parameter leaves (means, scales,
    quats, opacity, rgb, sem_w) and example target tensors that fix the
    shapes.  ``step(h_rgb, h_depth, h_sem)`` takes pinned host tensors and
    returns the slot index whose ``grads`` / ``loss`` hold the result once
    the stream reaches it; ``loss_host(slot)`` is the pinned host copy of the
    loss, valid after ``synchronize()``.
    """

    def __init__(self, rast: raster.Rasterizer, g: raster.Gaussians, cam, params, t_rgb, t_depth, t_sem=None):
        self.rast, self.g, self.cam, self.params = rast, g, cam, list(params)
        dev = t_rgb.device
        self.slots = []
        for _ in range(2):
            self.slots.append((torch.empty_like(t_rgb), torch.empty_like(t_depth),
                               None if t_sem is None else torch.empty_like(t_sem)))
            for dst, src in zip(self.slots[-1], (t_rgb, t_depth, t_sem)):
                if dst is not None:
                    dst.copy_(src)
        self.copy_stream = torch.cuda.Stream(device=dev)
        self.filled = [torch.cuda.Event() for _ in range(2)]
        self.consumed = [torch.cuda.Event() for _ in range(2)]
        self.loss_pinned = [torch.empty((), dtype=torch.float32).pin_memory() for _ in range(2)]
        self.graphs, self.loss, self.grads = [], [], []
        for s in range(2):
            graph, (loss, grads) = self._capture(s)
            self.graphs.append(graph)
            self.loss.append(loss)
            self.grads.append(grads)
        self.count = 0

    def _step_body(self, s):
        tr, td, ts = self.slots[s]
        loss = raster.render_l1(self.rast, self.g, self.cam, tr, td, ts, *self.params, check=False)
        grads = torch.autograd.grad(loss, self.params)
        return loss, grads

    def _capture(self, s):
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(2):
                self._step_body(s)
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            out = self._step_body(s)
        return graph, out

    def step(self, h_rgb, h_depth, h_sem=None) -> int:
        """Enqueues one step on the current stream; returns its slot."""
        s = self.count & 1
        self.count += 1
        cur = torch.cuda.current_stream()
        tr, td, ts = self.slots[s]
        with torch.cuda.stream(self.copy_stream):
            # the slot's previous graph must be done with it
            self.copy_stream.wait_event(self.consumed[s])
            tr.copy_(h_rgb, non_blocking=True)
            td.copy_(h_depth, non_blocking=True)
            if ts is not None and h_sem is not None:
                ts.copy_(h_sem, non_blocking=True)
            self.filled[s].record(self.copy_stream)
        cur.wait_event(self.filled[s])
        self.graphs[s].replay()
        self.consumed[s].record(cur)
        self.loss_pinned[s].copy_(self.loss[s].detach(), non_blocking=True)
        return s

    def loss_host(self, s) -> float:
        return float(self.loss_pinned[s])
