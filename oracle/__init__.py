"""CPU oracle for exact FPS / RadiusFPS -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The library's product path never does, and the
two share no code: the oracle is plain C in ``rfps_oracle.c`` (compiled with
``-ffp-contract=off``, no fast-math) plus a numpy brute force here.

Functions and the passages they follow:

* ``fps``            -- plain FPS, Alg. 1 / Sec. 3.1 (pinned: hand-worked
                        examples, brute force, invariants, closed forms).
* ``fps_bruteforce`` -- the argmax-min definition of Sec. 3.1 recomputed from
                        scratch every step (numpy, tiny inputs only).
* ``radiusfps``      -- the CPU RadiusFPS of Sec. 3.2-3.4 with the prune / skip
                        switches of Tab. ablation (pinned: identical to ``fps``).
* ``voxelize``       -- the voxel grid of Sec. 3.2 (pinned: closed-form cells,
                        containment, brute force).
* ``fps_f64``        -- FP64 square-root-domain FPS, information only
                        (pinned by the hand-worked examples).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import sysconfig

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rfps_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_rfps.so")

OK, EINVAL, ENONFINITE, ENOMEM = 0, 1, 2, 3


class OracleError(RuntimeError):
    pass


def build(src: str = _SRC, out: str = _LIB, extra: tuple = ()) -> str:
    """Compile the oracle with gcc (-O2 -ffp-contract=off, OpenMP when available)."""
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            "-std=c11", *extra, src, "-o", out, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       stdout=subprocess.PIPE, stderr=subprocess.PIPE)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    return out


def _declare(lib):
    i64p = ctypes.POINTER(ctypes.c_int64)
    f32p = ctypes.POINTER(ctypes.c_float)
    f64p = ctypes.POINTER(ctypes.c_double)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.oracle_fps.argtypes = [f32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, i64p, f32p,
                               ctypes.c_int]
    lib.oracle_fps.restype = ctypes.c_int
    lib.oracle_radiusfps.argtypes = [f32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     i64p, i64p]
    lib.oracle_radiusfps.restype = ctypes.c_int
    lib.oracle_voxelize.argtypes = [f32p, ctypes.c_int64, ctypes.c_int, f32p, u32p]
    lib.oracle_voxelize.restype = ctypes.c_int
    lib.oracle_fps_f64.argtypes = [f32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, i64p, f64p]
    lib.oracle_fps_f64.restype = ctypes.c_int
    lib.oracle_has_openmp.argtypes = []
    lib.oracle_has_openmp.restype = ctypes.c_int
    return lib


_lib = None


def load(path: str | None = None):
    """Load (building if needed) the oracle library; a path loads another build of it."""
    global _lib
    if path is not None:
        return _declare(ctypes.CDLL(path))
    if _lib is None:
        if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            build()
        _lib = _declare(ctypes.CDLL(_LIB))
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _pts(points) -> np.ndarray:
    p = np.ascontiguousarray(points, dtype=np.float32)
    if p.ndim != 2 or p.shape[1] != 3:
        raise ValueError("points must have shape (N, 3)")
    return p


def _check(rc):
    if rc != OK:
        raise OracleError({EINVAL: "invalid argument", ENONFINITE: "non-finite coordinate",
                           ENOMEM: "out of memory"}.get(rc, f"error {rc}"))


def fps(points, m: int, start: int = 0, threads: int = 1, return_d2: bool = False, lib=None):
    """Plain FPS (Alg. 1): int64 indices of the m samples in selection order."""
    lib = lib or load()
    p = _pts(points)
    out = np.empty(m, dtype=np.int64)
    d2 = np.empty(p.shape[0], dtype=np.float32) if return_d2 else None
    rc = lib.oracle_fps(_ptr(p, ctypes.c_float), p.shape[0], m, start, _ptr(out, ctypes.c_int64),
                        _ptr(d2, ctypes.c_float) if d2 is not None else None, threads)
    _check(rc)
    return (out, d2) if return_d2 else out


def radiusfps(points, m: int, start: int = 0, n_vox: int = 16, prune: bool = True,
              skip: bool = True, radius_mode: int = 0, lib=None):
    """CPU RadiusFPS (Sec. 3.2-3.4): (indices, stats dict)."""
    lib = lib or load()
    p = _pts(points)
    out = np.empty(m, dtype=np.int64)
    st = np.zeros(6, dtype=np.int64)
    rc = lib.oracle_radiusfps(_ptr(p, ctypes.c_float), p.shape[0], m, start, n_vox, int(prune),
                              int(skip), radius_mode, _ptr(out, ctypes.c_int64),
                              _ptr(st, ctypes.c_int64))
    _check(rc)
    keys = ("voxel_tests", "voxels_pruned", "points_visited", "points_skipped", "points_updated",
            "active_voxels")
    return out, dict(zip(keys, (int(x) for x in st)))


def voxelize(points, n_vox: int, lib=None):
    """Voxel grid of Sec. 3.2: (grid dict with min, max, L; uint32 voxel id per point)."""
    lib = lib or load()
    p = _pts(points)
    grid = np.empty(7, dtype=np.float32)
    vid = np.empty(p.shape[0], dtype=np.uint32)
    rc = lib.oracle_voxelize(_ptr(p, ctypes.c_float), p.shape[0], n_vox, _ptr(grid, ctypes.c_float),
                             _ptr(vid, ctypes.c_uint32))
    _check(rc)
    return {"min": grid[0:3].copy(), "max": grid[3:6].copy(), "L": np.float32(grid[6])}, vid


def fps_f64(points, m: int, start: int = 0, lib=None):
    """FP64 square-root-domain FPS (information only): (indices, coverage radius per step)."""
    lib = lib or load()
    p = _pts(points)
    out = np.empty(m, dtype=np.int64)
    cov = np.empty(m, dtype=np.float64)
    rc = lib.oracle_fps_f64(_ptr(p, ctypes.c_float), p.shape[0], m, start, _ptr(out, ctypes.c_int64),
                            _ptr(cov, ctypes.c_double))
    _check(rc)
    return out, cov


def openmp_threads(lib=None) -> int:
    """OpenMP threads the oracle would use (0 if it was built without OpenMP)."""
    return int((lib or load()).oracle_has_openmp())


def sq_dist_np(points: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Canonical FP32 squared distance of every point to s, one rounded numpy op at a time."""
    p = np.asarray(points, dtype=np.float32)
    s = np.asarray(s, dtype=np.float32)
    dx = p[:, 0] - s[0]
    dy = p[:, 1] - s[1]
    dz = p[:, 2] - s[2]
    return (dx * dx + dy * dy) + dz * dz


def fps_bruteforce(points, m: int, start: int = 0) -> np.ndarray:
    """Sec. 3.1 argmax-min definition, recomputed from scratch at every step.

    s_j = argmax_p min_{s in S_{j-1}} d2(p, s), ties to the smallest index
    (np.argmax returns the first maximum).  O(N * M^2): tiny inputs only.
    """
    p = _pts(points)
    sel = [int(start)]
    for _ in range(1, m):
        d = np.stack([sq_dist_np(p, p[s]) for s in sel]).min(axis=0)
        sel.append(int(np.argmax(d)))
    return np.array(sel, dtype=np.int64)
