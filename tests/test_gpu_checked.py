"""Parity cases against the bounds-checked build of the library.

The test builds librfps_checked.so (-DRFPS_CHECKED: every index the
sampling kernel takes from data -- a record's point range, a super-record or
record list entry, the record that owns a candidate -- is checked, and an
out-of-range one records RFPS_EBOUNDS instead of being used) and runs, in a
child process that loads it, the launch shapes and paths of the library:
shared-memory records with all points resident, partly resident, the
hierarchical path, ties, ragged batches and incremental sampling.  Every
call must end with status 0 and the indices must equal the oracle's.
"""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import cloudgen, oracle
import paper_2606_06255_gb300 as rf
assert rf._lib.LIB_PATH.endswith("librfps_checked.so"), rf._lib.LIB_PATH
dev = lambda p: torch.from_numpy(np.ascontiguousarray(p, dtype=np.float32)).cuda()
lat = np.stack(np.meshgrid(*[np.arange(12)] * 3, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
cases = [
    ("room_20k_c16_t128", cloudgen.room_cloud(20000, seed=1), 3000, {"cluster": 16, "threads": 128}),
    ("room_20k_c16_t256", cloudgen.room_cloud(20000, seed=2), 3000, {"cluster": 16}),
    ("lidar_60k_c1_t512", cloudgen.lidar_cloud(60000, seed=3), 3000, {"cluster": 1, "threads": 512}),
    ("lidar_30k_c4_chunk256", cloudgen.lidar_cloud(30000, seed=4), 3000, {"cluster": 4, "chunk": 256}),
    ("uniform_60k_hier_c1", cloudgen.uniform_cloud(60000, seed=5), 800, {"cluster": 1, "chunk": 32, "n_vox": 40}),
    ("uniform_60k_hier_c2", cloudgen.uniform_cloud(60000, seed=6), 800, {"cluster": 2, "chunk": 32, "n_vox": 48}),
    ("lattice_ties_c8", lat, 1500, {"cluster": 8}),
]
for name, pts, m, o in cases:
    got = rf.fps(dev(pts), m, 0, opts=o, check=True).cpu().numpy()
    assert np.array_equal(got, oracle.fps(pts, m, 0, threads=0)), name
clouds = [cloudgen.room_cloud(9000, seed=7), cloudgen.lidar_cloud(15000, seed=8), cloudgen.uniform_cloud(4000, seed=9)]
sizes = [c.shape[0] for c in clouds]; ms = [n // 5 for n in sizes]
ws = torch.empty(rf.batch_workspace_size(sum(sizes), 3, max(sizes), {"cluster": 4}), dtype=torch.uint8, device="cuda")
out, oo = rf.fps_batched(dev(np.concatenate(clouds)), sizes, ms, [0, 0, 0], opts={"cluster": 4}, workspace=ws)
assert rf.status(ws) == 0
out = out.cpu().numpy()
for b, c in enumerate(clouds):
    assert np.array_equal(out[oo[b]:oo[b + 1]], oracle.fps(c, ms[b], 0, threads=0)), b
pts = cloudgen.uniform_cloud(60000, seed=10)
ix = rf.Index(dev(pts), opts={"cluster": 1, "n_vox": 40, "chunk": 32})
got = np.concatenate([ix.sample(700, 0).cpu().numpy(), ix.sample_more(500).cpu().numpy()])
assert np.array_equal(got, oracle.fps(pts, 1200, 0, threads=0))
ix.free()
print("checked build: all cases clean")
'''


def _checked_library():
    import importlib.util
    spec = importlib.util.spec_from_file_location("rfps_build_script",
                                                  os.path.join(ROOT, "paper_2606_06255_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build(checked=True)


def test_checked_build_runs_clean():
    lib = _checked_library()
    env = dict(os.environ, RFPS_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, stdout=subprocess.PIPE,
                       stderr=subprocess.PIPE, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    assert "all cases clean" in r.stdout
