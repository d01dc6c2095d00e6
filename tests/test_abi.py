"""The C ABI library loads and exports what include/rfps.h declares (no GPU calls)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rfps.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(rfps_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__._builder().build()
    from paper_2606_06255_gb300 import _lib
    return _lib.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    for code in range(8):
        s = lib.rfps_status_str(code)
        assert s and s != b"unknown status"
    assert lib.rfps_status_str(99) == b"unknown status"
    assert lib.rfps_version() >= 1


def test_defaults(lib):
    from paper_2606_06255_gb300 import Opts
    o = Opts()
    d = o.as_dict()
    assert d["prune"] == 1 and d["skip"] == 1 and d["radius_mode"] == 0
    assert d["n_vox"] == 0 and d["cluster"] == 0 and d["threads"] == 0 and d["chunk"] == 0


def test_resolved_defaults(lib):
    import paper_2606_06255_gb300 as rf
    small, big = rf.resolved_opts(1000), rf.resolved_opts(100000)
    assert small["cluster"] == 1 and big["cluster"] == 16
    assert big["threads"] == 256 and big["chunk"] == 128 and big["prune"] == 1 and big["skip"] == 1
    assert rf.resolved_opts(100000, {"cluster": 4, "threads": 512})["cluster"] == 4
    with pytest.raises(rf.RfpsError):
        rf.resolved_opts(100, {"chunk": 3})


def test_workspace_sizes_are_host_only(lib):
    from paper_2606_06255_gb300 import Opts
    s1 = lib.rfps_fps_workspace_size(1000, None)
    s2 = lib.rfps_fps_workspace_size(100000, None)
    assert 0 < s1 < s2
    assert s2 >= 100000 * 16      # at least the sorted float4 points
    assert lib.rfps_fps_workspace_size(0, None) == 0
    assert lib.rfps_fps_host_workspace_size(1000, None) > s1
    assert lib.rfps_batch_workspace_size(10000, 4, 5000, None) > 0
    assert lib.rfps_batch_workspace_size(10000, 0, 5000, None) == 0
    assert lib.rfps_plain_workspace_size(1000, 1) > 0
    bad = Opts(chunk=100)            # not a power of two
    assert lib.rfps_fps_workspace_size(1000, ctypes.byref(bad)) == 0
    bad = Opts(cluster=3)
    assert lib.rfps_fps_workspace_size(1000, ctypes.byref(bad)) == 0
    bad = Opts(threads=1024)
    assert lib.rfps_fps_workspace_size(1000, ctypes.byref(bad)) == 0


def test_argument_errors_need_no_device(lib):
    """Invalid arguments are rejected on the host before anything touches CUDA."""
    EINVAL = 1
    fake = ctypes.c_void_p(256)
    assert lib.rfps_fps(None, 10, 3, 0, fake, None, fake, 1 << 20, None) == EINVAL
    assert lib.rfps_fps(fake, 10, 11, 0, fake, None, fake, 1 << 20, None) == EINVAL   # M > N
    assert lib.rfps_fps(fake, 10, 0, 0, fake, None, fake, 1 << 20, None) == EINVAL    # M = 0
    assert lib.rfps_fps(fake, 10, 3, 10, fake, None, fake, 1 << 20, None) == EINVAL   # start >= N
    assert lib.rfps_fps(fake, 10, 3, -1, fake, None, fake, 1 << 20, None) == EINVAL
    assert lib.rfps_fps(fake, 10, 3, 0, fake, None, ctypes.c_void_p(257), 1 << 20, None) == EINVAL  # misaligned
    assert lib.rfps_fps(fake, 1 << 31, 3, 0, fake, None, fake, 1 << 40, None) == EINVAL
    assert lib.rfps_plain_fps(fake, 10, 3, 0, fake, 7, fake, 1 << 20, None) == EINVAL   # no variant 7
    assert lib.rfps_fps_batched(fake, 10, None, 1, fake, fake, 10, fake, None, fake, 1 << 20, None) == EINVAL
    assert lib.rfps_index_sample(None, 1, 0, fake, None) == EINVAL
    assert lib.rfps_status_read(None, None) == EINVAL
    sink = ctypes.c_void_p(256)
    assert lib.rfps_bandwidth_probe(2, fake, 4096, 1, sink, None, None, None) == EINVAL       # no kind 2
    assert lib.rfps_bandwidth_probe(0, fake, 4096, 0, sink, None, None, None) == EINVAL       # reps = 0
    assert lib.rfps_bandwidth_probe(1, None, 0, 1 << 21, sink, None, None, None) == EINVAL    # reps > 2^20
    assert lib.rfps_bandwidth_probe(0, None, 4096, 1, sink, None, None, None) == EINVAL       # no buffer
    assert lib.rfps_bandwidth_probe(0, ctypes.c_void_p(264), 4096, 1, sink, None, None, None) == EINVAL
    assert lib.rfps_bandwidth_probe(0, fake, 4100, 1, sink, None, None, None) == EINVAL       # not x16
    assert lib.rfps_bandwidth_probe(1, None, 0, 1, None, None, None, None) == EINVAL          # no sink
    assert lib.rfps_bandwidth_probe(1, None, 0, 1, ctypes.c_void_p(260), None, None, None) == EINVAL
    lib.rfps_index_free(None)


def test_launch_counter_starts_at_zero_without_gpu(lib):
    assert lib.rfps_launch_count() >= 0


def test_noalloc_capacity_is_pinned(lib):
    """rfps_fps_noalloc's fixed 64 MiB scratch holds a 725,440-point cloud with default options and
    not one point more; beyond it the call is rejected on the host (nothing is launched)."""
    cap = 64 << 20
    assert lib.rfps_fps_workspace_size(725440, None) <= cap < lib.rfps_fps_workspace_size(725441, None)
    ENOMEM = 3
    fake = ctypes.c_void_p(256)
    assert lib.rfps_fps_noalloc(fake, 725441, 10, 0, fake, None, None) == ENOMEM
