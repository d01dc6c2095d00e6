"""Ragged batches of clouds in one persistent launch, replayed from a CUDA graph.

A BatchSampler owns static device buffers for one batch shape (cloud sizes,
sample counts, start indices): the concatenated points, the per-cloud
offsets, the workspace and the output.  The whole call (voxel index build of
every cloud plus the persistent sampling kernel, whose cluster groups take
clouds largest first from a device work queue) is captured once into a CUDA
graph and replayed, so a step costs one graph launch.
"""

from __future__ import annotations

import numpy as np
import torch

from . import _lib


class BatchSampler:
    def __init__(self, sizes, ms, starts=None, opts=None, device=None, graph: bool = True):
        self.sizes = [int(s) for s in sizes]
        self.ms = [int(x) for x in ms]
        self.starts = [int(x) for x in (starts if starts is not None else [0] * len(self.sizes))]
        if not self.sizes or min(self.sizes) < 1:
            raise ValueError("every cloud needs at least one point")
        if any(m < 1 or m > n for m, n in zip(self.ms, self.sizes)):
            raise ValueError("1 <= M_b <= N_b for every cloud")
        self.device = torch.device(device if device is not None else "cuda")
        self.opts = opts
        total = sum(self.sizes)
        self.points = torch.zeros((total, 3), dtype=torch.float32, device=self.device)
        self.meta = _lib._batch_meta(self.sizes, self.ms, self.starts, self.device)
        self.offsets = self.meta[3]
        self.out_offsets = self.meta[4]
        nbytes = _lib.batch_workspace_size(total, len(self.sizes), max(self.sizes), opts)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.out = torch.empty(int(self.out_offsets[-1]), dtype=torch.int64, device=self.device)
        self._graph = None
        self.kernels_per_run = None
        if graph:
            self._capture()

    def _launch(self, stream=None):
        d_off, d_ooff, d_st, off, ooff, max_n = self.meta
        _lib._check(_lib.lib().rfps_fps_batched(
            self.points.data_ptr(), self.points.shape[0], d_off.data_ptr(), len(self.sizes), d_ooff.data_ptr(),
            d_st.data_ptr(), max_n, self.out.data_ptr(), _lib._opts(self.opts), self.workspace.data_ptr(),
            self.workspace.numel(), _lib._stream(stream)), "rfps_fps_batched")

    def _capture(self):
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            self._launch(s)          # first call outside capture: kernel attributes, device check
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        before = _lib.launch_count()
        with torch.cuda.graph(g, stream=s):
            self._launch(s)
        self.kernels_per_run = _lib.launch_count() - before   # kernel nodes each replay launches
        torch.cuda.current_stream(self.device).wait_stream(s)
        self._graph = g

    def load(self, clouds):
        """Copy a list of (N_b, 3) arrays / tensors (the batch shape) into the static input buffer."""
        for b, c in enumerate(clouds):
            t = torch.as_tensor(np.ascontiguousarray(c, dtype=np.float32)) if not isinstance(c, torch.Tensor) else c
            self.points[int(self.offsets[b]):int(self.offsets[b + 1])].copy_(t, non_blocking=True)

    def run(self):
        """Sample every cloud of the loaded batch (asynchronous); returns the output buffer."""
        if self._graph is not None:
            self._graph.replay()
        else:
            self._launch()
        return self.out

    def split(self, out=None):
        """Per-cloud index arrays (host) from the output buffer."""
        o = (self.out if out is None else out).cpu().numpy()
        return [o[int(self.out_offsets[b]):int(self.out_offsets[b + 1])] for b in range(len(self.sizes))]

    def status(self) -> int:
        return _lib.status(self.workspace)
