"""Serving loop with continuous batching for RadiusFPS requests.

Requests (a cloud, M, start) arrive over time.  The scheduler admits waiting
requests whenever a stream slot is free and the device-memory budget has
room.  Everything admitted in the same scheduling pass is launched as one
micro-batch: the points are copied to the device, the batched call builds
each cloud's voxel index on the device and samples all clouds in one
persistent launch, and the indices are copied back.  Micro-batches on
different streams overlap on the GPU, so clouds that arrive while others
are running start as soon as memory and a slot free up, without waiting for
the running batch to finish.  Results are bit-identical to sampling each
cloud alone: every cloud's indices depend only on its own points.

The GPU work sits behind a small executor interface (mem_needed / launch /
done / results) so the scheduling logic can be exercised on the CPU with a
simulated executor.

Failures degrade service instead of stopping it: a micro-batch whose launch
raises (an allocation or API error) or whose results report a device error
(a timed-out wait, a non-finite coordinate) releases its slot and memory,
and its requests are queued again: from a batch of several each runs alone
next (so one bad request cannot take its batch-mates down), and a request
that fails on its own is retried up to `max_retries` times, then reported
as failed.  A request may carry a queueing deadline (dropped as expired if
not admitted in time) and a cancellation time (dropped if still queued then).

Kept indices and follow-up requests (incremental sampling, Sec. 3.3-3.4): a
request with keep=True leaves its cloud's voxel index and FPS state (every
point's distance, the records' Dist_v keys, the last sample) on the device
after it is served; a later request with more_of=<that rid> asks for m more
samples of the same sequence and is served from that state, without the
points travelling again and without repeating the first samples' work.  A
kept index counts against the memory budget until a follow-up without
keep=True consumes it or the run ends.  A follow-up waits while its base
request is still queued or running, and fails if the base was not kept.

Size-aware routing: an executor may ask for some requests to run alone
(alone(r) -> True; the GPU executor does so for clouds above `tail_n` points,
which it launches with their own launch shape, e.g. a cluster of CTAs
instead of one CTA), so that the few largest clouds, which set the latency
tail, get more of the GPU each.
"""

from __future__ import annotations

import collections
import statistics
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    points: np.ndarray      # (N, 3) float32 (or a pinned host tensor)
    m: int
    start: int = 0
    deadline: float | None = None    # seconds after arrival by which it must be admitted
    cancel_at: float | None = None   # the client withdraws it at this time if still queued
    attempts: int = 0                # launches that failed so far
    keep: bool = False               # keep the device index and FPS state for follow-ups
    more_of: int | None = None       # continue the sequence of this earlier (kept) request by m samples


@dataclass
class Completed:
    rid: int
    arrival: float
    admitted: float
    finished: float
    batch_size: int
    indices: np.ndarray
    samples: int = 0        # len(indices), kept when the indices themselves are dropped

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class Report:
    completed: list = field(default_factory=list)
    rejected: list = field(default_factory=list)     # can never fit the memory budget
    failed: list = field(default_factory=list)       # (rid, reason) after the retries ran out
    expired: list = field(default_factory=list)      # not admitted before their deadline
    cancelled: list = field(default_factory=list)    # withdrawn while queued
    makespan: float = 0.0
    offered_rate: float = 0.0
    window: tuple = (0.0, 0.0)       # first and last arrival
    max_inflight_batches: int = 0
    peak_mem: int = 0
    followups: int = 0               # follow-up requests served from a kept index

    def summary(self) -> dict:
        lat = sorted(c.latency for c in self.completed)
        q = lambda p: lat[min(len(lat) - 1, int(round(p * (len(lat) - 1))))] if lat else None
        n = len(self.completed)
        # completions per second over the middle half of the arrival window (steady state:
        # equal to the offered rate when the server keeps up)
        t0, t1 = self.window
        a, b = t0 + 0.25 * (t1 - t0), t0 + 0.75 * (t1 - t0)
        steady = sum(1 for c in self.completed if a <= c.finished <= b)
        return {
            "steady_clouds_per_s": steady / (b - a) if b > a else None,
            "requests_completed": n,
            "requests_rejected": len(self.rejected),
            "requests_failed": len(self.failed),
            "requests_expired": len(self.expired),
            "requests_cancelled": len(self.cancelled),
            "offered_clouds_per_s": self.offered_rate,
            "achieved_clouds_per_s": n / self.makespan if self.makespan > 0 else None,
            "p50_latency_ms": 1e3 * q(0.50) if lat else None,
            "p99_latency_ms": 1e3 * q(0.99) if lat else None,
            "mean_latency_ms": 1e3 * statistics.mean(lat) if lat else None,
            "mean_batch_size": statistics.mean(c.batch_size for c in self.completed) if n else None,
            "max_inflight_batches": self.max_inflight_batches,
            "peak_device_bytes": self.peak_mem,
            "followups_served": self.followups,
            "samples_per_s": sum(c.samples for c in self.completed) / self.makespan if self.makespan else None,
        }


def merge_reports(reports) -> "Report":
    """One report for a request stream served by several servers (one per GPU, each with a share of
    the requests): outcomes concatenated; the arrival window, offered rate and makespan taken over
    the whole stream; peak device memory summed over the servers."""
    out = Report()
    live = [r for r in reports if r.window != (0.0, 0.0) or r.completed]
    for r in reports:
        out.completed += r.completed
        out.rejected += r.rejected
        out.failed += r.failed
        out.expired += r.expired
        out.cancelled += r.cancelled
        out.max_inflight_batches = max(out.max_inflight_batches, r.max_inflight_batches)
        out.peak_mem += r.peak_mem
        out.followups += r.followups
    if live:
        t0 = min(r.window[0] for r in live)
        t1 = max(r.window[1] for r in live)
        out.window = (t0, t1)
        n = len(out.completed) + len(out.rejected) + len(out.failed) + len(out.expired) + len(out.cancelled)
        out.offered_rate = (n - 1) / (t1 - t0) if t1 > t0 else float("inf")
        out.makespan = max(r.window[0] + r.makespan for r in live) - t0
    return out


class Server:
    def __init__(self, executor, mem_budget: int, max_inflight: int = 4, max_batch: int = 16,
                 poll_s: float = 2e-4, max_retries: int = 1):
        if max_inflight < 1 or max_batch < 1 or mem_budget <= 0 or max_retries < 0:
            raise ValueError("bad server limits")
        self.ex = executor
        self.budget = int(mem_budget)
        self.max_inflight = int(max_inflight)
        self.max_batch = int(max_batch)
        self.poll_s = poll_s
        self.max_retries = int(max_retries)

    def run(self, requests, clock=time.perf_counter, sleep=time.sleep) -> Report:
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        rep = Report()
        if reqs:
            span = reqs[-1].arrival - reqs[0].arrival
            rep.offered_rate = (len(reqs) - 1) / span if span > 0 else float("inf")
            rep.window = (reqs[0].arrival, reqs[-1].arrival)
        t0 = clock()
        i = 0
        queue = collections.deque()
        inflight = {}            # slot -> (handle, batch, admitted_at, mem)
        free_slots = list(range(self.max_inflight))[::-1]
        mem_used = 0
        last_finish = 0.0
        alone = set()            # rids that run in a batch of their own after a batch failure
        kept = {}                # rid -> device bytes of its kept index
        busy = set()             # kept rids a follow-up is running on
        settled = set()          # rids that completed or were dropped (a follow-up of one not kept fails)
        ex_alone = getattr(self.ex, "alone", None)

        def runs_alone(r):
            return r.keep or r.more_of is not None or r.rid in alone or bool(ex_alone and ex_alone(r))

        def release(rid):
            nonlocal mem_used
            if rid in kept:
                mem_used -= kept.pop(rid)
                self.ex.release(rid)

        def requeue(batch, reason):
            # a failed micro-batch: its requests go back to the head of the queue to run alone; one
            # that failed alone spends a retry, and fails for good when they run out.  A follow-up
            # is not retried: the kept state it started from is no longer trusted.
            for r in reversed(batch):
                if len(batch) > 1:
                    alone.add(r.rid)
                    queue.appendleft(r)
                    continue
                r.attempts += 1
                if r.more_of is not None:
                    busy.discard(r.more_of)
                    release(r.more_of)
                    rep.failed.append((r.rid, reason))
                    settled.add(r.rid)
                elif r.attempts > self.max_retries:
                    rep.failed.append((r.rid, reason))
                    settled.add(r.rid)
                else:
                    queue.appendleft(r)

        while i < len(reqs) or queue or inflight:
            now = clock() - t0
            progressed = False
            while i < len(reqs) and reqs[i].arrival <= now:
                queue.append(reqs[i])
                i += 1
                progressed = True
            if any(r.deadline is not None or r.cancel_at is not None for r in queue):
                keep = collections.deque()
                for r in queue:
                    if r.cancel_at is not None and now >= r.cancel_at:
                        rep.cancelled.append(r.rid)
                        settled.add(r.rid)
                    elif r.deadline is not None and now > r.arrival + r.deadline:
                        rep.expired.append(r.rid)
                        settled.add(r.rid)
                    else:
                        keep.append(r)
                progressed = progressed or len(keep) != len(queue)
                queue = keep
            for slot in list(inflight):
                handle, batch, t_adm, mem = inflight[slot]
                if self.ex.done(handle):
                    t_done = clock() - t0
                    try:
                        results = self.ex.results(handle)
                    except Exception as e:   # a device error reported with the results
                        results = None
                        requeue(batch, f"results: {e}")
                    mem_used -= mem
                    if results is not None:
                        for r, idx in zip(batch, results):
                            rep.completed.append(Completed(r.rid, r.arrival, t_adm, t_done, len(batch), idx, len(idx)))
                            settled.add(r.rid)
                            if r.more_of is not None:      # the kept state moved on to this request
                                rep.followups += 1
                                busy.discard(r.more_of)
                                held = kept.pop(r.more_of, 0)
                                if r.keep:
                                    kept[r.rid] = held
                                else:
                                    mem_used -= held
                                    self.ex.release(r.rid)
                            elif r.keep:
                                kept[r.rid] = self.ex.kept_bytes(r.rid)
                                mem_used += kept[r.rid]
                        last_finish = max(last_finish, t_done)
                    free_slots.append(slot)
                    del inflight[slot]
                    progressed = True
            while queue and free_slots:
                # a follow-up whose base is still queued or running waits; one whose base was not
                # kept (finished without keep, failed, dropped) fails now
                blocked = []
                while queue and queue[0].more_of is not None and (queue[0].more_of not in kept
                                                                   or queue[0].more_of in busy):
                    r = queue.popleft()
                    if r.more_of in settled and r.more_of not in kept:
                        rep.failed.append((r.rid, "follow-up of a request whose index was not kept"))
                        settled.add(r.rid)
                        progressed = True
                    else:
                        blocked.append(r)
                if not queue:
                    queue.extendleft(reversed(blocked))
                    break
                head = queue[0]
                if self.ex.mem_needed([head]) > self.budget:
                    rep.rejected.append(queue.popleft().rid)     # can never fit
                    settled.add(head.rid)
                    queue.extendleft(reversed(blocked))
                    progressed = True
                    continue
                batch = []
                while queue and len(batch) < self.max_batch:
                    if batch and (runs_alone(queue[0]) or runs_alone(batch[0])):
                        break
                    if batch and queue[0].more_of is not None:
                        break
                    need = self.ex.mem_needed(batch + [queue[0]])
                    if mem_used + need > self.budget:
                        break
                    batch.append(queue.popleft())
                queue.extendleft(reversed(blocked))
                if not batch:
                    break                                        # wait for memory to free up
                need = self.ex.mem_needed(batch)
                slot = free_slots.pop()
                try:
                    handle = self.ex.launch(batch, slot)
                except Exception as e:       # allocation or API error: the slot stays free
                    free_slots.append(slot)
                    requeue(batch, f"launch: {e}")
                    progressed = True
                    break
                inflight[slot] = (handle, batch, clock() - t0, need)
                if batch[0].more_of is not None:
                    busy.add(batch[0].more_of)
                mem_used += need
                rep.peak_mem = max(rep.peak_mem, mem_used)
                rep.max_inflight_batches = max(rep.max_inflight_batches, len(inflight))
                progressed = True
            if not progressed:
                wait = self.poll_s
                if i < len(reqs) and not inflight and not queue:
                    wait = max(0.0, min(reqs[i].arrival - now, 0.01))
                sleep(wait)
        for rid in list(kept):       # kept indices live as long as the run
            release(rid)
        rep.makespan = last_finish - (reqs[0].arrival if reqs else 0.0)
        return rep


class GpuExecutor:
    """Runs micro-batches with the batched C ABI call, one CUDA stream per slot.

    Per launch: each cloud's points are copied host -> device (pinned host
    tensors are copied asynchronously; numpy arrays are staged through a
    pinned buffer), the per-cloud offsets, sample counts and starts go up in
    one pinned buffer, the batched call samples every cloud, and the indices
    come back into a pinned buffer.  All of it is ordered on the slot's stream.
    """

    def __init__(self, n_slots: int, opts=None, device=None, tail_opts=None, tail_n: int | None = None):
        import ctypes

        import torch

        from . import _lib
        self.torch = torch
        self.lib = _lib
        self.ctypes = ctypes
        self.device = torch.device(device if device is not None else "cuda")
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(n_slots)]
        self.opts = opts
        self._opts = _lib.Opts(**opts) if opts else None
        # clouds of tail_n points or more run alone with their own launch shape
        self.tail_n = tail_n if tail_opts is not None else None
        self.tail_opts = tail_opts
        self._tail_opts = _lib.Opts(**tail_opts) if tail_opts else None
        self.kept = {}        # rid -> Index kept on the device for follow-up requests

    def alone(self, r) -> bool:
        return self.tail_n is not None and r.more_of is None and r.points.shape[0] >= self.tail_n

    def _route(self, batch):
        if len(batch) == 1 and self.alone(batch[0]):
            return self.tail_opts, self._tail_opts
        return self.opts, self._opts

    def mem_needed(self, batch) -> int:
        if not batch:
            return 0
        if batch[0].more_of is not None:           # the kept index already holds the cloud
            return 8 * batch[0].m + 4096
        opts, _ = self._route(batch)
        sizes = [r.points.shape[0] for r in batch]
        total = sum(sizes)
        if batch[0].keep:
            ws = self.lib.host_workspace_size(total, opts)   # the index's own memory (points included)
        else:
            ws = self.lib.batch_workspace_size(total, len(batch), max(sizes), opts)
        return total * 12 + ws + 8 * sum(r.m for r in batch) + 4096

    def kept_bytes(self, rid) -> int:
        ix = self.kept.get(rid)
        return ix.nbytes if ix is not None else 0

    def release(self, rid):
        ix = self.kept.pop(rid, None)
        if ix is not None:
            ix.free()

    def _launch_kept(self, r, s):
        """keep=True: build the cloud's index on the device and take the first m samples from it;
        more_of: the next m samples from the kept index of an earlier request."""
        torch = self.torch
        with torch.cuda.stream(s):
            held = []
            if r.more_of is not None:
                ix = self.kept[r.more_of]
                out = ix.sample_more(r.m, stream=s)
            else:
                src = r.points
                if not isinstance(src, torch.Tensor):
                    src = torch.from_numpy(np.ascontiguousarray(src, dtype=np.float32)).pin_memory()
                pts = src.to(self.device, non_blocking=True)
                ix = self.lib.Index(pts, opts=self.opts, stream=s)   # copies the points on the stream
                out = ix.sample(r.m, r.start, stream=s)
                held = [src, pts]
            host_out = torch.empty(r.m, dtype=torch.int64, pin_memory=True)
            host_out.copy_(out, non_blocking=True)
            host_st = torch.empty(1, dtype=torch.int32, pin_memory=True)
            ix.status_into(host_st, stream=s)
            ev = torch.cuda.Event()
            ev.record(s)
        return {"event": ev, "host_out": host_out, "host_st": host_st, "ooff": np.array([0, r.m]),
                "index": ix, "rid": r.rid, "base": r.more_of, "keep": (out, *held)}

    def launch(self, batch, slot):
        torch = self.torch
        s = self.streams[slot]
        if len(batch) == 1 and (batch[0].keep or batch[0].more_of is not None):
            return self._launch_kept(batch[0], s)
        opts, c_opts = self._route(batch)
        b = len(batch)
        sizes = [int(r.points.shape[0]) for r in batch]
        ms = [int(r.m) for r in batch]
        total, mtotal = sum(sizes), sum(ms)
        meta = torch.empty(3 * b + 2, dtype=torch.int64, pin_memory=True)
        mv = meta.numpy()
        mv[0] = 0
        mv[1:b + 1] = np.cumsum(sizes)
        mv[b + 1] = 0
        mv[b + 2:2 * b + 2] = np.cumsum(ms)
        mv[2 * b + 2:] = [int(r.start) for r in batch]
        staged = []
        with torch.cuda.stream(s):
            pts = torch.empty((total, 3), dtype=torch.float32, device=self.device)
            o = 0
            for r in batch:
                src = r.points
                if not isinstance(src, torch.Tensor):
                    src = torch.from_numpy(np.ascontiguousarray(src, dtype=np.float32)).pin_memory()
                    staged.append(src)
                pts[o:o + src.shape[0]].copy_(src, non_blocking=True)
                o += src.shape[0]
            dmeta = meta.to(self.device, non_blocking=True)
            ws = torch.empty(self.lib.batch_workspace_size(total, b, max(sizes), opts), dtype=torch.uint8,
                             device=self.device)
            out = torch.empty(mtotal, dtype=torch.int64, device=self.device)
            base = dmeta.data_ptr()
            self.lib._check(self.lib.lib().rfps_fps_batched(
                pts.data_ptr(), total, base, b, base + 8 * (b + 1), base + 16 * (b + 1), max(sizes),
                out.data_ptr(), self.ctypes.byref(c_opts) if c_opts is not None else None,
                ws.data_ptr(), ws.numel(), s.cuda_stream), "rfps_fps_batched")
            host_out = torch.empty(mtotal, dtype=torch.int64, pin_memory=True)
            host_out.copy_(out, non_blocking=True)
            # the workspace's status word (its first 4 bytes) comes back with the indices, so that
            # results() reads it without a synchronising call
            host_st = torch.empty(1, dtype=torch.int32, pin_memory=True)
            host_st.copy_(ws[:4].view(torch.int32), non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        ooff = np.concatenate([[0], np.cumsum(ms)])
        # keep every buffer alive until the event completes
        return {"event": ev, "host_out": host_out, "host_st": host_st, "ooff": ooff,
                "keep": (meta, dmeta, pts, ws, out, staged)}

    def done(self, handle) -> bool:
        return handle["event"].query()

    def results(self, handle):
        st = int(handle["host_st"][0])   # copied back with the indices; the event has fired
        if st != 0:
            if "index" in handle and handle["base"] is None:
                handle["index"].free()   # a new index that failed is not kept
            raise RuntimeError(f"device status {st}")
        if "index" in handle:            # the index (new, or moved on by a follow-up) is kept under this rid
            if handle["base"] is not None:
                self.kept.pop(handle["base"], None)
            self.kept[handle["rid"]] = handle["index"]
        o, ooff = handle["host_out"].numpy(), handle["ooff"]
        return [o[ooff[b]:ooff[b + 1]].copy() for b in range(len(ooff) - 1)]


def poisson_workload(n_requests: int, rate: float, lo: int = 20000, hi: int = 1200000, ratio: float = 0.125,
                     pool: int = 48, seed: int = 0, pinned: bool = False):
    """Poisson arrivals of room-like / LiDAR-like clouds with N log-uniform in [lo, hi] and M = N * ratio.

    A pool of distinct seeded clouds (drawn from the same size and kind
    distribution) is generated once and requests cycle through it, which keeps
    host memory bounded for long runs.  pinned=True keeps the pool in pinned
    host memory (requests then arrive in page-locked buffers).
    """
    import math

    import cloudgen

    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=pool))).astype(np.int64)
    clouds = []
    for k, n in enumerate(sizes):
        if k % 2 == 0:
            clouds.append(cloudgen.room_cloud(int(n), seed=seed * 1000 + k))
        else:
            clouds.append(cloudgen.lidar_cloud(int(n), seed=seed * 1000 + k, scan_seed=k // 2 % 4))
    if pinned:
        import torch
        clouds = [torch.from_numpy(c).pin_memory() for c in clouds]
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    pick = rng.integers(0, pool, size=n_requests)
    return [Request(i, float(t[i]), clouds[pick[i]], max(1, int(clouds[pick[i]].shape[0] * ratio)), 0)
            for i in range(n_requests)]


def main(argv=None):
    import argparse
    import json

    ap = argparse.ArgumentParser(description="Serve a Poisson stream of RadiusFPS requests on one GPU")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=200.0, help="offered arrivals per second")
    ap.add_argument("--slots", type=int, default=32, help="micro-batches in flight (one stream each)")
    ap.add_argument("--max-batch", type=int, default=8)
    ap.add_argument("--mem-gb", type=float, default=32.0, help="device-memory budget for admitted work")
    ap.add_argument("--opts", default='{"cluster": 1, "threads": 512}')
    ap.add_argument("--warmup", type=int, default=16)
    args = ap.parse_args(argv)
    reqs = poisson_workload(args.requests + args.warmup, args.rate, pinned=True)
    ex = GpuExecutor(args.slots, opts=json.loads(args.opts))
    server = Server(ex, mem_budget=int(args.mem_gb * (1 << 30)), max_inflight=args.slots, max_batch=args.max_batch)
    server.run(reqs[:args.warmup])        # warm-up: kernel attributes, allocator pools
    timed = [Request(r.rid, r.arrival - reqs[args.warmup].arrival, r.points, r.m, r.start)
             for r in reqs[args.warmup:]]
    rep = server.run(timed)
    out = rep.summary()
    out.update({"requests": args.requests, "rate": args.rate, "slots": args.slots, "max_batch": args.max_batch,
                "opts": json.loads(args.opts), "mem_budget_gb": args.mem_gb})
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
