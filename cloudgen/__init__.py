"""Seeded synthetic point clouds shaped like the paper's workloads.

The paper evaluates on real scans (S3DIS / ScanNet indoor rooms, SemanticKITTI
rotating-LiDAR scenes, Sec. 5.1 and Sec. 5.6).  None of those datasets is
available here, so these generators stand in for them with the same kind of
shape, size, density and structure:

* ``uniform``  -- i.i.d. points in the unit cube (the small plain-FPS case).
* ``room``     -- an indoor room: floor, ceiling and four walls of a 10 x 8 x 3 m
                  box plus 12 axis-aligned boxes standing on the floor, points
                  spread over the surfaces in proportion to their area, with
                  isotropic Gaussian noise (sigma 5 mm).
* ``lidar``    -- an accumulated rotating-LiDAR scan: 64 beams between -25 and
                  +3 degrees elevation, 1,875 azimuth steps per sweep, 10 sweeps
                  from poses 1 m apart, ray-cast against a ground plane and 200
                  boxes within 80 m, range noise sigma 2 cm; rays without a hit
                  inside 80 m are dropped, so density falls with range.
* ``batch``    -- ragged batches of room-like and LiDAR-like clouds with sizes
                  log-uniform in [lo, hi].

This module holds only input generation: no step of the sampling method is
computed here.  Both the CPU oracle tests and the CUDA path draw their inputs
from it.  Every generator is a pure function of its seed (numpy PCG64).
"""

from __future__ import annotations

import math
import os
from dataclasses import dataclass

import numpy as np

__all__ = [
    "uniform_cloud",
    "room_cloud",
    "lidar_scan",
    "lidar_cloud",
    "ragged_batch",
    "serving_requests",
    "Cloud",
    "workload",
]


def uniform_cloud(n: int, seed: int = 0) -> np.ndarray:
    """``n`` points i.i.d. uniform in [0, 1)^3, float32, shape (n, 3)."""
    rng = np.random.default_rng(seed)
    return rng.random((n, 3), dtype=np.float32)


def _room_surfaces(rng: np.random.Generator, room=(10.0, 8.0, 3.0), n_boxes: int = 12):
    """Axis-aligned rectangles (origin, edge u, edge v) making up a furnished room."""
    X, Y, Z = room
    rects = []
    # floor, ceiling
    rects.append(((0.0, 0.0, 0.0), (X, 0.0, 0.0), (0.0, Y, 0.0)))
    rects.append(((0.0, 0.0, Z), (X, 0.0, 0.0), (0.0, Y, 0.0)))
    # four walls
    rects.append(((0.0, 0.0, 0.0), (X, 0.0, 0.0), (0.0, 0.0, Z)))
    rects.append(((0.0, Y, 0.0), (X, 0.0, 0.0), (0.0, 0.0, Z)))
    rects.append(((0.0, 0.0, 0.0), (0.0, Y, 0.0), (0.0, 0.0, Z)))
    rects.append(((X, 0.0, 0.0), (0.0, Y, 0.0), (0.0, 0.0, Z)))
    for _ in range(n_boxes):
        sx, sy, sz = rng.uniform(0.3, 2.0, size=3)
        sz = min(sz, Z - 0.05)
        x0 = rng.uniform(0.0, X - sx)
        y0 = rng.uniform(0.0, Y - sy)
        # five visible faces (no bottom face)
        rects.append(((x0, y0, sz), (sx, 0.0, 0.0), (0.0, sy, 0.0)))          # top
        rects.append(((x0, y0, 0.0), (sx, 0.0, 0.0), (0.0, 0.0, sz)))         # -y side
        rects.append(((x0, y0 + sy, 0.0), (sx, 0.0, 0.0), (0.0, 0.0, sz)))    # +y side
        rects.append(((x0, y0, 0.0), (0.0, sy, 0.0), (0.0, 0.0, sz)))         # -x side
        rects.append(((x0 + sx, y0, 0.0), (0.0, sy, 0.0), (0.0, 0.0, sz)))    # +x side
    o = np.array([r[0] for r in rects], dtype=np.float64)
    u = np.array([r[1] for r in rects], dtype=np.float64)
    v = np.array([r[2] for r in rects], dtype=np.float64)
    area = np.linalg.norm(np.cross(u, v), axis=1)
    return o, u, v, area


def room_cloud(n: int, seed: int = 0, noise: float = 0.005) -> np.ndarray:
    """Indoor-room-like cloud of exactly ``n`` float32 points (metres)."""
    rng = np.random.default_rng(seed)
    o, u, v, area = _room_surfaces(rng)
    # area-proportional allocation of the n points, exact total
    face = rng.choice(len(area), size=n, p=area / area.sum())
    a = rng.random(n)
    b = rng.random(n)
    pts = o[face] + a[:, None] * u[face] + b[:, None] * v[face]
    pts += rng.normal(0.0, noise, size=pts.shape)
    return pts.astype(np.float32)


def _ray_cast(origin, az, elev, boxes_lo, boxes_hi, max_range):
    """Nearest hit distance of each (azimuth, elevation) ray against z=0 and the boxes.

    Rays are laid out azimuth-major, shape (len(az), len(elev)).  Each box is
    tested only against the azimuth steps inside the angular sector it spans
    as seen from ``origin`` (boxes never contain the origin by construction).
    Returns (t, dirs) with t = inf where nothing is hit within ``max_range``.
    """
    ce, se = np.cos(elev), np.sin(elev)
    dirs = np.stack([
        ce[None, :] * np.cos(az)[:, None],
        ce[None, :] * np.sin(az)[:, None],
        np.broadcast_to(se[None, :], (az.shape[0], elev.shape[0])),
    ], axis=2)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(dirs[..., 2] < 0.0, -origin[2] / dirs[..., 2], np.inf)
        inv = 1.0 / dirs
    n_az = az.shape[0]
    step = 2.0 * math.pi / n_az
    a0 = az[0]
    for lo, hi in zip(boxes_lo, boxes_hi):
        cx = np.array([lo[0], hi[0], hi[0], lo[0]]) - origin[0]
        cy = np.array([lo[1], lo[1], hi[1], hi[1]]) - origin[1]
        ang = np.arctan2(cy, cx)
        # angular sector of the footprint, unwrapped around its first corner
        rel = np.mod(ang - ang[0] + math.pi, 2.0 * math.pi) - math.pi
        amin, amax = ang[0] + rel.min(), ang[0] + rel.max()
        i0 = int(math.floor((amin - a0) / step)) - 1
        i1 = int(math.ceil((amax - a0) / step)) + 1
        idx = np.arange(i0, i1 + 1) % n_az
        iv = inv[idx]
        t1 = (lo[None, None, :] - origin[None, None, :]) * iv
        t2 = (hi[None, None, :] - origin[None, None, :]) * iv
        with np.errstate(invalid="ignore"):
            tn = np.nanmax(np.minimum(t1, t2), axis=2)
            tf = np.nanmin(np.maximum(t1, t2), axis=2)
        hit = (tn <= tf) & (tn > 0.0)
        t[idx] = np.minimum(t[idx], np.where(hit, tn, np.inf))
    t[t > max_range] = np.inf
    return t, dirs


def lidar_scan(seed: int = 0, beams: int = 64, az_steps: int = 1875, sweeps: int = 10,
               n_boxes: int = 200, max_range: float = 80.0, height: float = 1.73,
               noise: float = 0.02) -> np.ndarray:
    """Full accumulated rotating-LiDAR scan (about 1.2M float32 points for the defaults)."""
    cache = _cache_path(f"lidar_{seed}_{beams}_{az_steps}_{sweeps}_{n_boxes}.npy")
    if cache and os.path.exists(cache):
        return np.load(cache)
    rng = np.random.default_rng(seed)
    # boxes: footprint centre uniform in a disc of radius max_range around the path,
    # standing on the ground, kept clear of the sensor path (|y| > 2.5 m or x outside path)
    lo, hi = [], []
    while len(lo) < n_boxes:
        r = max_range * math.sqrt(rng.random())
        th = rng.uniform(0.0, 2.0 * math.pi)
        cx, cy = 4.5 + r * math.cos(th), r * math.sin(th)
        sx, sy, sz = rng.uniform(0.5, 4.0, size=3)
        if abs(cy) < sy / 2 + 2.5 and -2.5 - sx / 2 < cx < 11.5 + sx / 2:
            continue
        lo.append((cx - sx / 2, cy - sy / 2, 0.0))
        hi.append((cx + sx / 2, cy + sy / 2, sz))
    boxes_lo = np.array(lo)
    boxes_hi = np.array(hi)
    elev = np.deg2rad(np.linspace(-25.0, 3.0, beams))
    out = []
    for k in range(sweeps):
        origin = np.array([float(k), 0.0, height])
        phase = rng.uniform(0.0, 2.0 * math.pi)
        az = phase + 2.0 * math.pi * np.arange(az_steps) / az_steps
        t, d = _ray_cast(origin, az, elev, boxes_lo, boxes_hi, max_range)
        t, d = t.ravel(), d.reshape(-1, 3)
        ok = np.isfinite(t)
        t = t[ok] + rng.normal(0.0, noise, size=int(ok.sum()))
        out.append(origin[None, :] + t[:, None] * d[ok])
    pts = np.concatenate(out).astype(np.float32)
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        np.save(cache, pts)
    return pts


def lidar_cloud(n: int | None = None, seed: int = 0, scan_seed: int | None = None) -> np.ndarray:
    """LiDAR-like cloud: the full scan (``n`` None) or a seeded random subset of ``n`` points."""
    full = lidar_scan(seed if scan_seed is None else scan_seed)
    if n is None or n >= full.shape[0]:
        return full
    rng = np.random.default_rng(seed + 7919)
    idx = np.sort(rng.choice(full.shape[0], size=n, replace=False))
    return np.ascontiguousarray(full[idx])


def _cache_path(name: str) -> str | None:
    root = os.environ.get("RFPS_CLOUD_CACHE")
    if root is None:
        root = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_cache")
    if root in ("", "0", "off"):
        return None
    return os.path.join(root, name)


@dataclass
class Cloud:
    points: np.ndarray   # (n, 3) float32
    m: int               # samples to draw
    start: int           # start index (original indexing)
    kind: str


def ragged_batch(n_clouds: int = 64, lo: int = 8000, hi: int = 200000, ratio: float = 0.25,
                 seed: int = 0, n_scans: int = 4) -> list[Cloud]:
    """Ragged batch: sizes round(exp(U[ln lo, ln hi])), alternating room / LiDAR-subset clouds."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_clouds))).astype(np.int64)
    clouds = []
    for b, n in enumerate(sizes):
        n = int(n)
        m = max(1, int(n * ratio))
        if b % 2 == 0:
            pts = room_cloud(n, seed=seed * 1000 + b)
            kind = "room"
        else:
            pts = lidar_cloud(n, seed=seed * 1000 + b, scan_seed=b // 2 % n_scans)
            kind = "lidar"
        clouds.append(Cloud(pts, m, 0, kind))
    return clouds


def serving_requests(n_requests: int, rate: float = 200.0, lo: int = 20000, hi: int = 1200000,
                     ratio: float = 0.125, seed: int = 0, n_scans: int = 4):
    """Poisson request stream: (arrival_time_s, Cloud) with log-uniform sizes, 50/50 kinds."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    sizes = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_requests))).astype(np.int64)
    kinds = rng.random(n_requests) < 0.5
    reqs = []
    for r in range(n_requests):
        n = int(sizes[r])
        if kinds[r]:
            pts = room_cloud(n, seed=seed * 100000 + r)
            kind = "room"
        else:
            pts = lidar_cloud(n, seed=seed * 100000 + r, scan_seed=r % n_scans)
            kind = "lidar"
        reqs.append((float(t[r]), Cloud(pts, max(1, int(n * ratio)), 0, kind)))
    return reqs


def workload(name: str, seed: int = 0):
    """The named workloads, as (list of Cloud, description)."""
    if name == "uniform4k":
        return [Cloud(uniform_cloud(4096, seed), 1024, 0, "uniform")], \
            "uniform N=4096 i.i.d. U[0,1)^3, M=1024, start 0"
    if name == "room100k":
        return [Cloud(room_cloud(100000, seed), 25000, 0, "room")], \
            "room-like N=100000, M=25000 (N/4), start 0"
    if name == "lidar1m":
        pts = lidar_cloud(None, seed)
        return [Cloud(pts, 16384, 0, "lidar")], \
            f"LiDAR-like accumulated scan N={pts.shape[0]}, M=16384, start 0"
    if name == "batch64":
        return ragged_batch(64, seed=seed), \
            "64 ragged clouds, N log-uniform [8000, 200000], alternating room/LiDAR, M=N/4"
    raise KeyError(name)
