"""Autotuner for the launch shape: cluster size, CTA threads, record chunk
(points per warp-sized record) and voxel resolution.

The sampling loop's per-iteration time is the cluster exchange plus the work
of the unpruned records, and the best trade-off depends on the cloud's size
and shape (Sec. 5.6.2 reports the same sensitivity to the voxel resolution
v).  The tuner times each candidate with CUDA events on representative
clouds (single cloud or a ragged batch) and keeps the fastest.  Results are
cached in a JSON file keyed by workload class and size bucket.  Every
candidate returns the same indices, so tuning never changes results.
"""

from __future__ import annotations

import json
import math
import os
import statistics

import torch

from . import _lib

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_cache",
                             "autotune.json")


def size_bucket(n: int) -> int:
    return int(round(math.log2(max(1, n))))


def key(kind: str, n: int, batch: int = 1) -> str:
    return f"{kind}:b{batch}:n{size_bucket(n)}"


# automatic voxel resolutions tried after the launch shape: nvox_scale / 100 * cbrt(N) bins per
# axis for every cloud (70 is the library default)
NVOX_SCALES = (35, 50, 70, 100, 140)


def default_candidates(batch: bool = False):
    """Launch shapes (cluster size, CTA threads, record chunk) the first stage times.

    Every cluster size the kernel supports is tried, with 128- and 256-thread CTAs and records of
    64, 128 or 256 points; 512-thread CTAs only in clusters of up to 4 (their exchange floor grows
    fastest with the cluster size)."""
    cands = []
    for cluster in (1, 2, 4, 8, 16):
        for threads in (128, 256, 512):
            if threads == 512 and cluster > 4:
                continue
            for chunk in ((64, 128, 256) if threads < 512 else (128,)):
                cands.append({"cluster": cluster, "threads": threads, "chunk": chunk})
    return cands


def candidate_space(batch: bool = False) -> str:
    """One-line description of what the tuner searches (for reports)."""
    return (f"stage 1: {len(default_candidates(batch))} launch shapes (cluster 1-16, threads 128/256/512, "
            f"chunk 64/128/256) at the automatic resolution; stage 2: the best 2 shapes x nvox_scale "
            f"{list(NVOX_SCALES)} (n_vox = scale/100 * cbrt(N) per cloud)")


def _time(fn, reps):
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def _two_stage(time_one, candidates, scales, keep: int = 2):
    """Stage 1 times every launch shape at the automatic resolution; stage 2 times the `keep`
    fastest shapes at each automatic-resolution scale.  Returns (best opts, rows sorted by time)."""
    rows = [(time_one(o), o) for o in candidates]
    rows.sort(key=lambda r: r[0])
    if not math.isfinite(rows[0][0]):
        raise RuntimeError("autotune: no candidate ran without a device error")
    for _, o in [r for r in rows if math.isfinite(r[0])][:keep]:
        for sc in scales:
            if sc == 70 or "n_vox" in o or "nvox_scale" in o:
                continue
            o2 = dict(o, nvox_scale=sc)
            rows.append((time_one(o2), o2))
    rows.sort(key=lambda r: r[0])
    return rows[0][1], rows


def tune_single(points: torch.Tensor, m: int, start: int = 0, candidates=None, reps: int = 3,
                scales=NVOX_SCALES):
    """Time launch shapes, then voxel resolutions, on one cloud; returns (best opts, [(ms, opts), ...]).
    Pass scales=() to time the candidates only."""
    n = points.shape[0]
    out = torch.empty(m, dtype=torch.int64, device=points.device)

    def time_one(o):
        ws = torch.empty(_lib.workspace_size(n, o), dtype=torch.uint8, device=points.device)
        ms = _time(lambda: _lib.fps(points, m, start, opts=o, workspace=ws, out=out), reps)
        # a shape the device could not run on this cloud (e.g. more records than one CTA can index)
        # records an error instead of sampling: never a candidate
        return ms if _lib.status(ws) == 0 else math.inf
    return _two_stage(time_one, candidates or default_candidates(False), scales)


def tune_batch(points: torch.Tensor, sizes, ms, starts=None, candidates=None, reps: int = 3, scales=NVOX_SCALES):
    """Time launch shapes, then voxel resolutions, on a ragged batch (one launch); returns (best opts, table)."""
    meta = _lib._batch_meta(sizes, ms, starts, points.device)

    def time_one(o):
        ws = torch.empty(_lib.batch_workspace_size(points.shape[0], len(sizes), max(sizes), o), dtype=torch.uint8,
                         device=points.device)
        t = _time(lambda: _lib.fps_batched(points, sizes, ms, starts, opts=o, workspace=ws, meta=meta), reps)
        return t if _lib.status(ws) == 0 else math.inf
    return _two_stage(time_one, candidates or default_candidates(True), scales)


def split_candidates(sizes, base_opts):
    """Size splits of a ragged batch to time against its single launch: the k largest clouds (k = 5,
    8, 10) in a launch of their own on 16- or 8-CTA clusters, the rest on 4-CTA clusters or with the
    single launch's options.  (Three tiers can be faster, but only when the largest tier's clusters
    start first, which stream priorities do not guarantee; they are not candidates.)"""
    order = sorted(sizes, reverse=True)
    o16 = {"cluster": 16, "threads": 256, "chunk": 128}
    o8 = {"cluster": 8, "threads": 256, "chunk": 128}
    o4 = {"cluster": 4, "threads": 256, "chunk": 128}

    def cut(k):   # the size at which the k largest clouds separate from the rest, or None
        return int(order[k - 1]) if 0 < k < len(order) and order[k] < order[k - 1] else None

    cands = []
    for k in (5, 8, 10):
        tail_n = cut(k)
        if tail_n is None:
            continue
        for tail_opts in (o16, o8):
            for rest in (o4, dict(base_opts or {})):
                cands.append((dict(rest), {"tail_n": tail_n, "tail_opts": tail_opts}))
    return cands


def tune_batch_split(clouds, sizes, ms, base_opts, reps: int = 3, candidates=None):
    """Time the single graph-replayed launch of a ragged batch against size splits (BatchSampler's
    split: the largest clouds in a concurrent launch of their own); returns ((opts, split or None),
    [(ms, opts, split), ...]) sorted by time.  Every candidate gives the same indices."""
    from . import batch

    def time_one(opts, split):
        bs = batch.BatchSampler(sizes, ms, opts=opts, split=split)
        bs.load(clouds)
        for _ in range(2):
            bs.run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            bs.run()
        e1.record()
        e1.synchronize()
        t = e0.elapsed_time(e1) / reps
        return t if bs.status() == 0 else math.inf

    table = [(time_one(dict(base_opts or {}), None), dict(base_opts or {}), None)]
    for opts, split in (candidates if candidates is not None else split_candidates(sizes, base_opts)):
        table.append((time_one(opts, split), opts, split))
    table.sort(key=lambda r: r[0])
    if not math.isfinite(table[0][0]):
        raise RuntimeError("no batch launch candidate ran without a device error")
    return (table[0][1], table[0][2]), table


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    if not os.path.exists(path):
        return {}
    with open(path) as fh:
        return json.load(fh)


def save(entry_key: str, opts: dict, table, path: str = DEFAULT_CACHE):
    cache = load_cache(path)
    cache[entry_key] = {"opts": opts, "table": [{"ms": round(ms, 4), "opts": o} for ms, o in table]}
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)


def best_opts(kind: str, n: int, batch: int = 1, path: str = DEFAULT_CACHE):
    """Cached best options for this workload class and size bucket, or None (library defaults)."""
    e = load_cache(path).get(key(kind, n, batch))
    return dict(e["opts"]) if e else None
