"""rfps_fps_noalloc: the entry point for callers that cannot allocate device memory.

Such callers (a real-time loop that cannot afford an allocation's implicit
synchronisation, a plug-in whose host application owns the device allocator)
pass only their input and output buffers; the library's scratch is a fixed
64 MiB array compiled into librfps.so.  These checks call it through the C ABI
and compare it index for index with rfps_fps on a caller workspace, on two
calls in a row, so that the second call also shows that the shared scratch
left by the first one does not leak into its result.  The file is named to be
collected last.
"""

import ctypes

import numpy as np
import pytest
import torch

import cloudgen

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2606_06255_gb300 import _lib as binding
    return binding.lib()


def _reference(lib, pts, m, start):
    n = pts.shape[0]
    ws = torch.empty(lib.rfps_fps_workspace_size(n, None), dtype=torch.uint8, device="cuda")
    out = torch.empty(m, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lib.rfps_fps(pts.data_ptr(), n, m, start, out.data_ptr(), None, ws.data_ptr(), ws.numel(), s) == 0
    assert lib.rfps_status_read(ws.data_ptr(), s) == 0
    return out.cpu().numpy()


def test_noalloc_matches_rfps_fps_twice():
    lib = _lib()
    s = torch.cuda.current_stream().cuda_stream
    # the third cloud (at most 4,096 points) takes the one-launch register-record path
    cases = [(cloudgen.room_cloud(60000, seed=41), 15000, 0),
             (cloudgen.lidar_cloud(25000, seed=42), 6000, 17),
             (cloudgen.room_cloud(3000, seed=46), 900, 3)]
    for pts_np, m, start in cases:
        pts = torch.from_numpy(pts_np).cuda()
        out = torch.full((m,), -1, dtype=torch.int64, device="cuda")
        rc = lib.rfps_fps_noalloc(pts.data_ptr(), pts.shape[0], m, start, out.data_ptr(), None, s)
        assert rc == 0, rc
        assert lib.rfps_noalloc_status_read(s) == 0     # no device-side error either
        ref = _reference(lib, pts, m, start)
        np.testing.assert_array_equal(out.cpu().numpy(), ref)


def test_noalloc_non_default_options():
    """Other options change the scratch layout; the result is still rfps_fps's."""
    from paper_2606_06255_gb300 import Opts
    lib = _lib()
    s = torch.cuda.current_stream().cuda_stream
    pts = torch.from_numpy(cloudgen.room_cloud(30000, seed=43)).cuda()
    m = 4000
    o = Opts(threads=128, chunk=256, cluster=4)
    out = torch.full((m,), -1, dtype=torch.int64, device="cuda")
    assert lib.rfps_fps_noalloc(pts.data_ptr(), pts.shape[0], m, 5, out.data_ptr(), ctypes.byref(o), s) == 0
    assert lib.rfps_noalloc_status_read(s) == 0
    np.testing.assert_array_equal(out.cpu().numpy(), _reference(lib, pts, m, 5))


def test_noalloc_reports_device_errors_then_recovers():
    """A non-finite coordinate is only visible on the device: the call returns 0 and the status read
    reports it; the next call on good points starts from a clean status word."""
    lib = _lib()
    s = torch.cuda.current_stream().cuda_stream
    bad = cloudgen.room_cloud(5000, seed=44)
    bad[1234, 1] = np.nan
    pts = torch.from_numpy(bad).cuda()
    out = torch.empty(100, dtype=torch.int64, device="cuda")
    assert lib.rfps_fps_noalloc(pts.data_ptr(), pts.shape[0], 100, 0, out.data_ptr(), None, s) == 0
    assert lib.rfps_noalloc_status_read(s) == 2      # RFPS_ENONFINITE
    good = torch.from_numpy(cloudgen.room_cloud(5000, seed=45)).cuda()
    assert lib.rfps_fps_noalloc(good.data_ptr(), good.shape[0], 100, 0, out.data_ptr(), None, s) == 0
    assert lib.rfps_noalloc_status_read(s) == 0
    np.testing.assert_array_equal(out.cpu().numpy(), _reference(lib, good, 100, 0))


def test_noalloc_small_cloud_error_then_recovery():
    """The same on the one-launch path for clouds of at most 4,096 points, whose kernel checks the
    points itself: the error is reported, and the next call's indices are rfps_fps's."""
    lib = _lib()
    s = torch.cuda.current_stream().cuda_stream
    bad = cloudgen.room_cloud(4000, seed=47)
    bad[3999, 2] = np.inf
    pts = torch.from_numpy(bad).cuda()
    out = torch.empty(500, dtype=torch.int64, device="cuda")
    assert lib.rfps_fps_noalloc(pts.data_ptr(), pts.shape[0], 500, 0, out.data_ptr(), None, s) == 0
    assert lib.rfps_noalloc_status_read(s) == 2      # RFPS_ENONFINITE
    for seed in (48, 49):
        good = torch.from_numpy(cloudgen.room_cloud(4000, seed=seed)).cuda()
        assert lib.rfps_fps_noalloc(good.data_ptr(), good.shape[0], 500, 7, out.data_ptr(), None, s) == 0
        assert lib.rfps_noalloc_status_read(s) == 0
        np.testing.assert_array_equal(out.cpu().numpy(), _reference(lib, good, 500, 7))


def test_noalloc_rejects_beyond_capacity():
    lib = _lib()
    fake = ctypes.c_void_p(256)
    ENOMEM, EINVAL = 3, 1
    assert lib.rfps_fps_noalloc(fake, 2_000_000, 10, 0, fake, None, None) == ENOMEM
    assert lib.rfps_fps_noalloc(fake, 1000, 1001, 0, fake, None, None) == EINVAL
