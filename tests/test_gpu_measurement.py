"""Measurement kernels behind the C ABI (needs a GB300): the sampling loop's
synchronisation floor and the on-chip bandwidth probes used as roofline
denominators.  The probes are checked to read every byte they claim to: after
an odd number of passes the XOR they fold into the sink equals the XOR of the
words they read, computed here on the host."""

import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rf():
    import paper_2606_06255_gb300 as rf
    return rf


def _probe(rf, kind, buf, nbytes, reps):
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    moved, sms = ctypes.c_int64(0), ctypes.c_int32(0)
    rc = rf.lib().rfps_bandwidth_probe(kind, buf.data_ptr() if buf is not None else None, nbytes, reps,
                                       sink.data_ptr(), ctypes.byref(moved), ctypes.byref(sms), None)
    assert rc == 0
    torch.cuda.synchronize()
    return int(sink.item()) & 0xFFFFFFFFFFFFFFFF, moved.value, sms.value


@pytest.mark.parametrize("nbytes", [4 << 20, (4 << 20) - 48, 16, 4096 + 16])
@pytest.mark.parametrize("reps", [1, 2, 3])
def test_l2_probe_reads_every_word(rf, nbytes, reps):
    g = np.random.default_rng(nbytes + reps)
    words = g.integers(0, 1 << 32, size=(4 << 20) // 4, dtype=np.uint64).astype(np.uint32)
    buf = torch.from_numpy(words.view(np.int32)).cuda()
    sink, moved, sms = _probe(rf, 0, buf, nbytes, reps)
    expect = int(np.bitwise_xor.reduce(words[: nbytes // 4])) if reps % 2 else 0
    assert sink == expect
    assert moved == nbytes * reps
    assert sms >= 1


@pytest.mark.parametrize("reps", [1, 2, 5])
def test_smem_probe_reads_every_word(rf, reps):
    sink, moved, sms = _probe(rf, 1, None, 0, reps)
    blocks = moved // (49152 * reps)
    assert moved == blocks * 49152 * reps and blocks % sms == 0
    b = np.arange(blocks, dtype=np.uint64)[:, None]
    i = np.arange(3072, dtype=np.uint64)[None, :]
    m32 = np.uint64(0xFFFFFFFF)
    w = (i ^ ((3 * i) & m32) ^ ((5 * i) & m32) ^ ((b * np.uint64(2654435761) + i) & m32)) & m32
    expect = int(np.bitwise_xor.reduce(w.ravel())) if reps % 2 else 0
    assert sink == expect


def test_bandwidths_are_plausible(rf):
    smem = rf.bandwidth_probe("smem")
    l2 = rf.bandwidth_probe("l2")
    # nominal shared-memory read rate is 128 B per clock per SM (265 GB/s per SM at 2.07 GHz)
    assert 30 < smem["gbs_per_sm"] < 600
    assert smem["sms"] == l2["sms"] >= 100
    assert 1000 < l2["gbs"] < 200000


@pytest.mark.parametrize("cluster,threads", [(1, 128), (2, 256), (16, 128), (16, 512)])
def test_sync_floor_runs_without_timeout(rf, cluster, threads):
    ms = rf.sync_floor(cluster, threads, 2000)
    assert 0 < ms < 1000
