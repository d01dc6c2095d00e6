"""Ragged batches of clouds in one persistent launch, replayed from a CUDA graph.

A BatchSampler owns static device buffers for one batch shape (cloud sizes,
sample counts, start indices): the concatenated points, the per-cloud
offsets, the workspace and the output.  The whole call (voxel index build of
every cloud plus the persistent sampling kernel, whose cluster groups take
clouds largest first from a device work queue) is captured once into a CUDA
graph and replayed, so a step costs one graph launch.

A ragged batch is bound by the latency of its largest clouds.  With
split={"tail_n": T, "tail_opts": {...}} the clouds of at least T points form a
second group, sampled by a launch of its own (for instance on larger clusters)
that runs beside the first group's on a second stream; split may also be a list
of such tiers, largest first ([{"tail_n": T1, "tail_opts": ...}, {"tail_n": T2,
...}]), each cloud going to the first tier it reaches.  All launches, the fork
and the join are captured in the same graph.  Each group's clouds sit
contiguously in the point buffer (largest tier first), so `rows` gives each
cloud's rows there; `split()` returns the indices in the caller's cloud order.
Without a split the sampler also exposes its single launch's `meta`, `offsets`,
`out_offsets` and `workspace`; with one, each of `groups` holds its own.
"""

from __future__ import annotations

import numpy as np
import torch

from . import _lib


class _Group:
    """One launch: clouds `ids` (caller order) at rows [row0, row0 + total) of the point buffer and
    output positions [out0, out0 + sum of their M)."""

    def __init__(self, ids, sizes, ms, starts, opts, row0, out0, device):
        self.ids = list(ids)
        self.opts = opts
        self.row0 = row0
        self.out0 = out0
        gs = [sizes[i] for i in self.ids]
        self.meta = _lib._batch_meta(gs, [ms[i] for i in self.ids], [starts[i] for i in self.ids], device)
        self.total = int(sum(gs))
        self.m_total = int(sum(ms[i] for i in self.ids))
        nbytes = _lib.batch_workspace_size(self.total, len(self.ids), max(gs), opts)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)


class BatchSampler:
    def __init__(self, sizes, ms, starts=None, opts=None, device=None, graph: bool = True, split=None):
        self.sizes = [int(s) for s in sizes]
        self.ms = [int(x) for x in ms]
        self.starts = [int(x) for x in (starts if starts is not None else [0] * len(self.sizes))]
        if not self.sizes or min(self.sizes) < 1:
            raise ValueError("every cloud needs at least one point")
        if any(m < 1 or m > n for m, n in zip(self.ms, self.sizes)):
            raise ValueError("1 <= M_b <= N_b for every cloud")
        self.device = torch.device(device if device is not None else "cuda")
        self.opts = opts
        tiers = [split] if isinstance(split, dict) else list(split or [])
        tiers = sorted((dict(t) for t in tiers), key=lambda t: -int(t["tail_n"]))
        self.split_spec = tiers or None
        b = len(self.sizes)
        left = list(range(b))
        plan = []
        for t in tiers:
            ids = [i for i in left if self.sizes[i] >= int(t["tail_n"])]
            left = [i for i in left if self.sizes[i] < int(t["tail_n"])]
            plan.append((ids, t["tail_opts"]))
        plan.append((left, opts))
        plan = [(ids, o) for ids, o in plan if ids]
        self.groups = []
        row = out = 0
        for ids, o in plan:
            g = _Group(ids, self.sizes, self.ms, self.starts, o, row, out, self.device)
            self.groups.append(g)
            row += g.total
            out += g.m_total
        # each cloud's rows in the point buffer and its range in the output, in the caller's order
        self.rows = [None] * b
        self.out_rows = [None] * b
        for g in self.groups:
            off, ooff = g.meta[3], g.meta[4]
            for k, i in enumerate(g.ids):
                self.rows[i] = (g.row0 + int(off[k]), g.row0 + int(off[k + 1]))
                self.out_rows[i] = (g.out0 + int(ooff[k]), g.out0 + int(ooff[k + 1]))
        total = sum(self.sizes)
        self.points = torch.zeros((total, 3), dtype=torch.float32, device=self.device)
        self.out = torch.empty(sum(self.ms), dtype=torch.int64, device=self.device)
        if len(self.groups) == 1:   # one group: the caller's order, the single launch's arrays
            self.meta = self.groups[0].meta
            self.offsets = self.meta[3]
            self.out_offsets = self.meta[4]
            self.workspace = self.groups[0].workspace
        # the smaller tiers run on streams of lower priority, so that the block scheduler starts the
        # larger tiers' clusters first when both wait for SMs (stream capture records the priority)
        self._side = ([torch.cuda.Stream(device=self.device, priority=0) for _ in self.groups[1:]]
                      if self.device.type == "cuda" else [])
        self._graph = None
        self.kernels_per_run = None
        if graph:
            self._capture()

    def _launch_group(self, g, stream):
        d_off, d_ooff, d_st, off, ooff, max_n = g.meta
        p = self.points[g.row0:g.row0 + g.total]
        o = self.out[g.out0:g.out0 + g.m_total]
        _lib._check(_lib.lib().rfps_fps_batched(
            p.data_ptr(), g.total, d_off.data_ptr(), len(g.ids), d_ooff.data_ptr(), d_st.data_ptr(), max_n,
            o.data_ptr(), _lib._opts(g.opts), g.workspace.data_ptr(), g.workspace.numel(), _lib._stream(stream)),
            "rfps_fps_batched")

    def _launch(self, stream=None):
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        for side in self._side:
            side.wait_stream(s)   # fork before any launch, so that the groups run side by side
        self._launch_group(self.groups[0], s)   # the largest tier first: its clusters take SMs first
        for g, side in zip(self.groups[1:], self._side):
            self._launch_group(g, side)
        for side in self._side:
            s.wait_stream(side)

    def _capture(self):
        s = torch.cuda.Stream(device=self.device, priority=-1 if len(self.groups) > 1 else 0)
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
            lo, hi = self.rows[b]
            self.points[lo:hi].copy_(t, non_blocking=True)

    def run(self):
        """Sample every cloud of the loaded batch (asynchronous); returns the output buffer."""
        if self._graph is not None:
            self._graph.replay()
        else:
            self._launch()
        return self.out

    def split(self, out=None):
        """Per-cloud index arrays (host), in the caller's cloud order, from the output buffer."""
        o = (self.out if out is None else out).cpu().numpy()
        return [o[lo:hi] for lo, hi in self.out_rows]

    def status(self) -> int:
        for g in self.groups:
            st = _lib.status(g.workspace)
            if st != 0:
                return st
        return 0
