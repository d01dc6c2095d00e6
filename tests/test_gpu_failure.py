"""The sampler's device-side failure path, exercised without faulting the GPU.

rfps_fps_lost_round drops every candidate message of one exchange iteration,
so each bounded wait of that iteration runs out (a flag that nothing sets).
The launch must end with RFPS_ETIMEOUT in the workspace's status word, every
CTA of the cluster must leave the kernel (the call returns and the stream
synchronises), and the next ordinary call on the same workspace must return
the oracle's indices with a clean status.  Covered for the shared-memory path
(records in shared memory, no CTA barrier per iteration: each warp leaves on
its own) and the hierarchical path (records in global memory: the CTA leaves
at its next barrier), at several cluster sizes and iterations.
"""

import numpy as np
import pytest
import torch

import cloudgen
import oracle

pytestmark = pytest.mark.gpu

ETIMEOUT, EINVAL = 5, 1


@pytest.fixture(scope="module")
def rf():
    import paper_2606_06255_gb300 as rf
    return rf


def _lost_round(rf, pts, m, start, opts, lost, spin=2000):
    lib = rf.lib()
    o = rf.Opts(**opts)
    import ctypes
    n = pts.shape[0]
    ws = torch.empty(rf.workspace_size(n, opts), dtype=torch.uint8, device="cuda")
    out = torch.empty(m, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    rc = lib.rfps_fps_lost_round(pts.data_ptr(), n, m, start, out.data_ptr(), ctypes.byref(o), ws.data_ptr(),
                                 ws.numel(), lost, spin, s)
    return rc, ws, out


@pytest.mark.parametrize("case", [
    ("room_20k_c4_t128", dict(cluster=4, threads=128), 1),
    ("room_20k_c16_t256", dict(cluster=16, threads=256), 137),
    ("room_20k_c2_t512", dict(cluster=2, threads=512), 1999),
    ("lidar_200k_c2_nv64_hier", dict(cluster=2, n_vox=64), 40),
], ids=lambda c: c[0])
def test_lost_exchange_round_times_out_then_workspace_recovers(rf, case):
    name, opts, lost = case
    pts_np = cloudgen.lidar_cloud(200000, seed=61) if name.startswith("lidar") else cloudgen.room_cloud(20000, seed=81)
    m = 2000
    pts = torch.from_numpy(pts_np).cuda()
    rc, ws, out = _lost_round(rf, pts, m, 3, opts, lost)
    assert rc == 0
    torch.cuda.synchronize()                   # every CTA left the kernel
    assert rf.status(ws) == ETIMEOUT
    # the same workspace, an ordinary call: clean status, exact indices
    got = rf.fps(pts, m, 3, opts=opts, workspace=ws)
    assert rf.status(ws) == 0
    np.testing.assert_array_equal(got.cpu().numpy(), oracle.fps(pts_np, m, 3, threads=0))


def test_lost_round_argument_checks(rf):
    pts = torch.from_numpy(cloudgen.room_cloud(5000, seed=82)).cuda()
    assert _lost_round(rf, pts, 100, 0, dict(cluster=1), 5)[0] == EINVAL      # no exchange on one CTA
    assert _lost_round(rf, pts, 100, 0, dict(cluster=4), 0)[0] == EINVAL      # iterations start at 1
    assert _lost_round(rf, pts, 100, 0, dict(cluster=4), 100)[0] == EINVAL    # beyond the last iteration
    assert _lost_round(rf, pts, 100, 0, dict(cluster=4), 5, spin=0)[0] == EINVAL
