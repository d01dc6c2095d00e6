"""ctypes binding of librfps.so (the C ABI in include/rfps.h).

Argument marshalling only: every step of sampling runs in the library's CUDA
kernels.  PyTorch provides device memory and the current stream.  There is no
CPU fallback: if librfps.so is missing or cannot be loaded, importing this
module raises.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# RFPS_LIBRARY selects another build of the same library (the bounds-checked test build)
LIB_PATH = os.environ.get("RFPS_LIBRARY") or os.path.join(_HERE, "librfps.so")

OK, EINVAL, ENONFINITE, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = range(7)


class RfpsError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        super().__init__(f"{what}: {_lib.rfps_status_str(int(status)).decode()} (status {int(status)})")


class Opts(ctypes.Structure):
    """rfps_opts: zero = automatic, except prune / skip (default 1)."""
    _fields_ = [("n_vox", ctypes.c_int32), ("cluster", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("chunk", ctypes.c_int32), ("prune", ctypes.c_int32), ("skip", ctypes.c_int32),
                ("radius_mode", ctypes.c_int32), ("counters", ctypes.c_int32), ("nvox_scale", ctypes.c_int32)]

    def __init__(self, **kw):
        super().__init__()
        _lib.rfps_opts_default(ctypes.byref(self))
        for k, v in kw.items():
            if k not in {f[0] for f in self._fields_}:
                raise TypeError(f"unknown option {k}")
            setattr(self, k, int(v))

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


class Counters(ctypes.Structure):
    _fields_ = [("voxel_tests", ctypes.c_uint64), ("voxels_pruned", ctypes.c_uint64),
                ("points_visited", ctypes.c_uint64), ("points_skipped", ctypes.c_uint64),
                ("points_updated", ctypes.c_uint64), ("iterations", ctypes.c_uint64),
                ("prune_violations", ctypes.c_uint64), ("skip_violations", ctypes.c_uint64),
                ("rounds", ctypes.c_uint64)]

    def as_dict(self):
        return {f[0]: int(getattr(self, f[0])) for f in self._fields_}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; g.build()\"`"
                          " (or python paper_2606_06255_gb300/build.py)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, sz, i64, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int64, ctypes.c_int32
    optp = ctypes.POINTER(Opts)
    st = ctypes.c_int
    sig = {
        "rfps_opts_default": (None, [optp]),
        "rfps_status_str": (ctypes.c_char_p, [ctypes.c_int]),
        "rfps_version": (ctypes.c_int, []),
        "rfps_opts_resolve": (st, [i64, optp, optp]),
        "rfps_launch_count": (i64, []),
        "rfps_fps_workspace_size": (sz, [i64, optp]),
        "rfps_fps": (st, [vp, i64, i64, i64, vp, optp, vp, sz, vp]),
        "rfps_fps_lost_round": (st, [vp, i64, i64, i64, vp, optp, vp, sz, i64, ctypes.c_uint32, vp]),
        "rfps_fps_host_workspace_size": (sz, [i64, optp]),
        "rfps_fps_host": (st, [vp, i64, i64, i64, vp, optp, vp, sz, vp]),
        "rfps_fps_noalloc": (st, [vp, i64, i64, i64, vp, optp, vp]),
        "rfps_noalloc_status_read": (st, [vp]),
        "rfps_batch_workspace_size": (sz, [i64, i64, i64, optp]),
        "rfps_fps_batched": (st, [vp, i64, vp, i64, vp, vp, i64, vp, optp, vp, sz, vp]),
        "rfps_plain_workspace_size": (sz, [i64, i64]),
        "rfps_plain_fps": (st, [vp, i64, i64, i64, vp, i32, vp, sz, vp]),
        "rfps_plain_fps_batched": (st, [vp, i64, vp, i64, vp, vp, i64, vp, i32, vp, sz, vp]),
        "rfps_bandwidth_probe": (st, [i32, vp, i64, i32, vp, ctypes.POINTER(i64), ctypes.POINTER(i32), vp]),
        "rfps_status_read": (st, [vp, vp]),
        "rfps_sync_floor": (st, [i32, i32, i64, vp, sz, vp]),
        "rfps_counters_read": (st, [vp, ctypes.POINTER(Counters), vp]),
        "rfps_index_build": (st, [vp, i64, optp, ctypes.POINTER(vp), vp]),
        "rfps_index_sample": (st, [vp, i64, i64, vp, vp]),
        "rfps_index_sample_more": (st, [vp, i64, vp, vp]),
        "rfps_index_distances": (st, [vp, vp, vp]),
        "rfps_index_bytes": (sz, [vp]),
        "rfps_index_status_copy": (st, [vp, vp, vp]),
        "rfps_index_free": (None, [vp]),
        "rfps_index_export": (st, [vp, ctypes.POINTER(i64), vp, vp, vp, vp, vp, vp, ctypes.POINTER(i32)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def lib():
    return _lib


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _check(status: int, what: str):
    if status != OK:
        raise RfpsError(status, what)


def _opts(opts):
    if opts is None:
        return None
    if isinstance(opts, Opts):
        return ctypes.byref(opts)
    return ctypes.byref(Opts(**opts))


def _points(points: torch.Tensor) -> torch.Tensor:
    if not isinstance(points, torch.Tensor) or not points.is_cuda:
        raise TypeError("points must be a CUDA tensor of shape (N, 3)")
    if points.dtype != torch.float32 or points.dim() != 2 or points.shape[1] != 3:
        raise TypeError("points must be float32 with shape (N, 3)")
    return points.contiguous()


def _workspace(nbytes: int, device, workspace=None) -> torch.Tensor:
    if nbytes == 0:
        raise RfpsError(EINVAL, "workspace size")
    if workspace is not None:
        if workspace.numel() * workspace.element_size() < nbytes or workspace.data_ptr() % 256:
            raise RfpsError(ENOMEM, "workspace")
        return workspace
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def workspace_size(n: int, opts=None) -> int:
    return int(_lib.rfps_fps_workspace_size(n, _opts(opts)))


def fps(points: torch.Tensor, m: int, start: int = 0, opts=None, workspace=None, stream=None,
        out: torch.Tensor | None = None, check: bool = False):
    """RadiusFPS: int64 indices (M,) of the samples, on the points' device.

    check=True synchronises and raises on a device-side error (e.g. a
    non-finite coordinate); otherwise the call is asynchronous.
    """
    p = _points(points)
    n = p.shape[0]
    ws = _workspace(workspace_size(n, opts), p.device, workspace)
    if out is None:
        out = torch.empty(m, dtype=torch.int64, device=p.device)
    s = _stream(stream)
    _check(_lib.rfps_fps(p.data_ptr(), n, m, start, out.data_ptr(), _opts(opts), ws.data_ptr(),
                         ws.numel(), s), "rfps_fps")
    if check:
        _check(_lib.rfps_status_read(ws.data_ptr(), s), "rfps_fps (device)")
    return out


def fps_host(points: np.ndarray, m: int, start: int = 0, opts=None, workspace=None, stream=None) -> np.ndarray:
    """RadiusFPS on host buffers (copies in and out inside the call, synchronises)."""
    p = np.ascontiguousarray(points, dtype=np.float32)
    if p.ndim != 2 or p.shape[1] != 3:
        raise TypeError("points must have shape (N, 3)")
    n = p.shape[0]
    nbytes = int(_lib.rfps_fps_host_workspace_size(n, _opts(opts)))
    ws = _workspace(nbytes, torch.device("cuda", torch.cuda.current_device()), workspace)
    out = np.empty(m, dtype=np.int64)
    _check(_lib.rfps_fps_host(p.ctypes.data, n, m, start, out.ctypes.data, _opts(opts), ws.data_ptr(), ws.numel(),
                              _stream(stream)), "rfps_fps_host")
    return out


def host_workspace_size(n: int, opts=None) -> int:
    return int(_lib.rfps_fps_host_workspace_size(n, _opts(opts)))


def _batch_meta(sizes, ms, starts, device):
    sizes = [int(x) for x in sizes]
    ms = [int(x) for x in ms]
    starts = [int(x) for x in (starts if starts is not None else [0] * len(sizes))]
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    ooff = np.zeros(len(sizes) + 1, dtype=np.int64)
    ooff[1:] = np.cumsum(ms)
    t = lambda a: torch.from_numpy(a).to(device)
    return t(off), t(ooff), t(np.array(starts, dtype=np.int64)), off, ooff, max(sizes)


def batch_workspace_size(total_n: int, b: int, max_n: int, opts=None) -> int:
    return int(_lib.rfps_batch_workspace_size(total_n, b, max_n, _opts(opts)))


def fps_batched(points: torch.Tensor, sizes, ms, starts=None, opts=None, workspace=None, stream=None, meta=None):
    """Ragged batch in one launch: returns (indices concatenated, host out-offsets)."""
    p = _points(points)
    if meta is None:
        meta = _batch_meta(sizes, ms, starts, p.device)
    d_off, d_ooff, d_st, off, ooff, max_n = meta
    b = len(off) - 1
    ws = _workspace(batch_workspace_size(p.shape[0], b, max_n, opts), p.device, workspace)
    out = torch.empty(int(ooff[-1]), dtype=torch.int64, device=p.device)
    _check(_lib.rfps_fps_batched(p.data_ptr(), p.shape[0], d_off.data_ptr(), b, d_ooff.data_ptr(), d_st.data_ptr(),
                                 max_n, out.data_ptr(), _opts(opts), ws.data_ptr(), ws.numel(), _stream(stream)),
           "rfps_fps_batched")
    return out, ooff


def plain_workspace_size(total_n: int, b: int = 1) -> int:
    return int(_lib.rfps_plain_workspace_size(total_n, b))


def plain_fps(points: torch.Tensor, m: int, start: int = 0, variant: int = 1, workspace=None, stream=None,
              out: torch.Tensor | None = None):
    """Plain O(N*M) GPU FPS baseline (variant 0 classic, 1 cluster, 2 whole GPU)."""
    p = _points(points)
    n = p.shape[0]
    ws = _workspace(plain_workspace_size(n), p.device, workspace)
    if out is None:
        out = torch.empty(m, dtype=torch.int64, device=p.device)
    _check(_lib.rfps_plain_fps(p.data_ptr(), n, m, start, out.data_ptr(), variant, ws.data_ptr(), ws.numel(),
                               _stream(stream)), "rfps_plain_fps")
    return out


def plain_fps_batched(points: torch.Tensor, sizes, ms, starts=None, variant: int = 1, workspace=None, stream=None,
                      meta=None):
    p = _points(points)
    if meta is None:
        meta = _batch_meta(sizes, ms, starts, p.device)
    d_off, d_ooff, d_st, off, ooff, max_n = meta
    b = len(off) - 1
    ws = _workspace(plain_workspace_size(p.shape[0], b), p.device, workspace)
    out = torch.empty(int(ooff[-1]), dtype=torch.int64, device=p.device)
    _check(_lib.rfps_plain_fps_batched(p.data_ptr(), p.shape[0], d_off.data_ptr(), b, d_ooff.data_ptr(),
                                       d_st.data_ptr(), max_n, out.data_ptr(), variant, ws.data_ptr(), ws.numel(),
                                       _stream(stream)), "rfps_plain_fps_batched")
    return out, ooff


def status(workspace: torch.Tensor, stream=None) -> int:
    return int(_lib.rfps_status_read(workspace.data_ptr(), _stream(stream)))


def counters(workspace: torch.Tensor, stream=None) -> dict:
    c = Counters()
    _check(_lib.rfps_counters_read(workspace.data_ptr(), ctypes.byref(c), _stream(stream)), "rfps_counters_read")
    return c.as_dict()


def bandwidth_probe(kind: str, nbytes: int = 64 << 20, reps: int | None = None, tries: int = 3,
                    stream=None) -> dict:
    """Read bandwidth of L2 ("l2": an `nbytes` buffer, small enough for L2, read with L2-only loads
    from every SM) or of shared memory ("smem": every resident CTA reads 48 KiB of its own), from
    the best of `tries` launches timed with CUDA events after a warm-up launch.  GB/s for the whole
    GPU and per SM."""
    k = {"l2": 0, "smem": 1}[kind]
    if reps is None:
        reps = 100 if k == 0 else 2000
    st = torch.cuda.current_stream() if stream is None else stream
    buf = torch.ones(nbytes // 4, dtype=torch.int32, device="cuda") if k == 0 else None
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    moved, sms = ctypes.c_int64(0), ctypes.c_int32(0)
    args = (k, buf.data_ptr() if buf is not None else None, nbytes if k == 0 else 0, reps, sink.data_ptr(),
            ctypes.byref(moved), ctypes.byref(sms), _stream(st))
    _check(_lib.rfps_bandwidth_probe(*args), "rfps_bandwidth_probe")
    best = float("inf")
    for _ in range(tries):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        _check(_lib.rfps_bandwidth_probe(*args), "rfps_bandwidth_probe")
        e1.record(st)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    gbs = moved.value / (best / 1e3) / 1e9
    return {"kind": kind, "gbs": gbs, "gbs_per_sm": gbs / max(1, sms.value), "bytes": moved.value, "ms": best,
            "sms": sms.value, "reps": reps, "buffer_bytes": nbytes if k == 0 else 49152}


def sync_floor(cluster: int, threads: int, iterations: int, stream=None) -> float:
    """Milliseconds of `iterations` rounds of the sampling loop's selection step alone (CUDA events)."""
    ws = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream() if stream is None else stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    _check(_lib.rfps_sync_floor(cluster, threads, iterations, ws.data_ptr(), ws.numel(), _stream(st)),
           "rfps_sync_floor")
    e0.record(st)
    _check(_lib.rfps_sync_floor(cluster, threads, iterations, ws.data_ptr(), ws.numel(), _stream(st)),
           "rfps_sync_floor")
    e1.record(st)
    e1.synchronize()
    if int(ws[128:132].view(torch.int32).item()) != 0:
        raise RfpsError(ETIMEOUT, "rfps_sync_floor (device)")
    return e0.elapsed_time(e1)


def resolved_opts(n: int, opts=None) -> dict:
    """The launch options the library uses for a cloud of n points (rfps_opts_resolve)."""
    o = Opts()
    _check(_lib.rfps_opts_resolve(n, _opts(opts), ctypes.byref(o)), "rfps_opts_resolve")
    return o.as_dict()


def launch_count() -> int:
    return int(_lib.rfps_launch_count())


class Index:
    """Device-resident spherical-voxel index of one cloud (rfps_index_*)."""

    def __init__(self, points: torch.Tensor, opts=None, stream=None):
        p = _points(points)
        self.n = p.shape[0]
        self.device = p.device
        h = ctypes.c_void_p()
        _check(_lib.rfps_index_build(p.data_ptr(), self.n, _opts(opts), ctypes.byref(h), _stream(stream)),
               "rfps_index_build")
        self._h = h

    @property
    def nbytes(self) -> int:
        return int(_lib.rfps_index_bytes(self._h))

    def sample(self, m: int, start: int = 0, stream=None, out: torch.Tensor | None = None) -> torch.Tensor:
        if self._h is None:
            raise RuntimeError("index freed")
        if out is None:
            out = torch.empty(m, dtype=torch.int64, device=self.device)
        _check(_lib.rfps_index_sample(self._h, m, start, out.data_ptr(), _stream(stream)), "rfps_index_sample")
        return out

    def sample_more(self, m_more: int, stream=None, out: torch.Tensor | None = None) -> torch.Tensor:
        """The next m_more samples of the sequence started by the last sample() call."""
        if self._h is None:
            raise RuntimeError("index freed")
        if out is None:
            out = torch.empty(m_more, dtype=torch.int64, device=self.device)
        _check(_lib.rfps_index_sample_more(self._h, m_more, out.data_ptr(), _stream(stream)),
               "rfps_index_sample_more")
        return out

    def distances(self, stream=None) -> torch.Tensor:
        """Every point's FP32 squared distance to the samples applied so far (all but the last)."""
        if self._h is None:
            raise RuntimeError("index freed")
        d2 = torch.empty(self.n, dtype=torch.float32, device=self.device)
        _check(_lib.rfps_index_distances(self._h, d2.data_ptr(), _stream(stream)), "rfps_index_distances")
        return d2

    def status_into(self, host: torch.Tensor, stream=None):
        """Enqueue a copy of the index's device status word into `host` (an int32 tensor of one
        element, pinned for an asynchronous copy); valid once the stream has passed this point."""
        if host.dtype != torch.int32 or host.numel() < 1 or host.is_cuda:
            raise TypeError("host must be a CPU int32 tensor")
        _check(_lib.rfps_index_status_copy(self._h, host.data_ptr(), _stream(stream)), "rfps_index_status_copy")

    def status(self, stream=None) -> int:
        """The index's device status word (synchronises the stream)."""
        h = torch.zeros(1, dtype=torch.int32)
        self.status_into(h, stream)
        (stream or torch.cuda.current_stream()).synchronize()
        return int(h[0])

    def export(self) -> dict:
        n = self.n
        R = ctypes.c_int64()
        _check(_lib.rfps_index_export(self._h, ctypes.byref(R), None, None, None, None, None, None, None),
               "rfps_index_export")
        r = R.value
        vid = np.empty(r, np.uint32)
        first = np.empty(r, np.uint32)
        cnt = np.empty(r, np.uint32)
        sph = np.empty((r, 4), np.float32)
        orig = np.empty(n, np.uint32)
        grid = np.empty(4, np.float32)
        nv = ctypes.c_int32()
        _check(_lib.rfps_index_export(self._h, ctypes.byref(R), vid.ctypes.data, first.ctypes.data, cnt.ctypes.data,
                                      sph.ctypes.data, orig.ctypes.data, grid.ctypes.data, ctypes.byref(nv)),
               "rfps_index_export")
        return {"voxel_id": vid, "first": first, "count": cnt, "sphere": sph, "sorted_orig": orig,
                "grid_min": grid[:3].copy(), "L": np.float32(grid[3]), "n_vox": nv.value}

    def free(self):
        if self._h is not None:
            _lib.rfps_index_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
