"""CUDA path vs the CPU oracle, element by element (needs a GB300).

Sample indices are integers decided by FP32 comparisons that both sides make
in the same precision, so the bar is bit-exact equality of every index.
"""

import numpy as np
import pytest
import torch

import cloudgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rf():
    import paper_2606_06255_gb300 as rf
    return rf


def dev(p):
    return torch.from_numpy(np.ascontiguousarray(p, dtype=np.float32)).cuda()


def gpu_fps(rf, pts, m, start=0, **opts):
    out = rf.fps(dev(pts), m, start, opts=opts or None, check=True)
    return out.cpu().numpy()


SMALL_CLOUDS = [
    ("uniform_4096", lambda: cloudgen.uniform_cloud(4096, seed=0), 1024, 0),
    ("uniform_ragged_5003", lambda: cloudgen.uniform_cloud(5003, seed=1), 1301, 17),
    ("room_20000", lambda: cloudgen.room_cloud(20000, seed=2), 5000, 0),
    ("lidar_30001", lambda: cloudgen.lidar_cloud(30001, seed=3), 3000, 123),
    ("grid_ties", lambda: np.array(np.meshgrid(*[np.arange(16)] * 3), dtype=np.float32).reshape(3, -1).T.copy(),
     1500, 0),
]


@pytest.mark.parametrize("name,make,m,start", SMALL_CLOUDS, ids=[c[0] for c in SMALL_CLOUDS])
def test_default_path_matches_oracle(rf, name, make, m, start):
    pts = make()
    ref = oracle.fps(pts, m, start, threads=0)
    np.testing.assert_array_equal(gpu_fps(rf, pts, m, start), ref)


OPT_GRID = [
    dict(cluster=1, threads=256, chunk=32, n_vox=4),
    dict(cluster=1, threads=512, chunk=4096, n_vox=64),
    dict(cluster=2, threads=512, chunk=64, n_vox=16),
    dict(cluster=4, threads=256, chunk=256, n_vox=32),
    dict(cluster=8, threads=256, chunk=128, n_vox=8),
    dict(cluster=16, threads=512, chunk=512, n_vox=48),
    dict(cluster=4, threads=512, chunk=256, n_vox=24, prune=0),
    dict(cluster=4, threads=512, chunk=256, n_vox=24, skip=0),
    dict(cluster=2, threads=512, chunk=256, n_vox=24, prune=0, skip=0),
    dict(cluster=2, threads=512, chunk=256, n_vox=20, radius_mode=1),
    dict(cluster=1, threads=128, chunk=64, n_vox=12),
    dict(cluster=16, threads=128, chunk=128, n_vox=24),
    dict(cluster=8, threads=128, chunk=32, n_vox=40),
    dict(cluster=1, threads=512, chunk=64, n_vox=12, prune=0),
    dict(cluster=16, threads=512, chunk=128, n_vox=24, skip=0),
    dict(n_vox=1),
    dict(n_vox=256, chunk=32),
]


@pytest.mark.parametrize("opts", OPT_GRID, ids=[str(o) for o in OPT_GRID])
def test_launch_shapes_and_switches(rf, opts):
    """Every cluster size, CTA size, record chunk, resolution and switch gives the same indices."""
    pts = cloudgen.room_cloud(12000, seed=11)
    ref = oracle.fps(pts, 3000, 5, threads=0)
    np.testing.assert_array_equal(gpu_fps(rf, pts, 3000, 5, **opts), ref)


def test_shared_memory_overflow_path(rf):
    """More records than one CTA holds in shared memory: the rest are read from global memory."""
    pts = cloudgen.uniform_cloud(60000, seed=12)
    ref = oracle.fps(pts, 2000, 0, threads=0)
    # chunk 32 and 40^3 cells -> ~ (cells + N/32) records on a single CTA
    np.testing.assert_array_equal(gpu_fps(rf, pts, 2000, 0, cluster=1, chunk=32, n_vox=40), ref)


@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 255, 257, 2047, 2049])
def test_tiny_and_ragged_sizes(rf, n):
    pts = cloudgen.uniform_cloud(n, seed=n)
    for m in sorted({1, min(n, 2), n // 2 or 1, n}):
        ref = oracle.fps(pts, m, n - 1)
        np.testing.assert_array_equal(gpu_fps(rf, pts, m, n - 1), ref)


def test_golden_examples(rf):
    import json
    import os
    import pins
    for case in json.load(open(os.path.join(pins.GOLDEN, "fps_hand_worked.json")))["cases"]:
        pts = np.array(case["points"], dtype=np.float32)
        if "points_bits" in case:
            pts = np.array(case["points_bits"], dtype=np.uint32).view(np.float32)
        for opts in ({}, {"n_vox": 2}, {"cluster": 2}):
            got = gpu_fps(rf, pts, case["m"], case["start"], **opts)
            assert got.tolist() == case["expected"], (case["name"], opts)
        for v in (0, 1, 2):
            got = rf.plain_fps(dev(pts), case["m"], case["start"], variant=v).cpu().numpy()
            assert got.tolist() == case["expected"], (case["name"], "plain", v)


def test_degenerate_clouds(rf):
    same = np.tile(np.array([[1.5, -2.0, 7.0]], np.float32), (1000, 1))
    np.testing.assert_array_equal(gpu_fps(rf, same, 10, 3), oracle.fps(same, 10, 3))
    dup = cloudgen.uniform_cloud(50, seed=4)[np.random.default_rng(0).integers(0, 50, size=3000)]
    np.testing.assert_array_equal(gpu_fps(rf, dup, 200, 0), oracle.fps(dup, 200, 0))
    flat = cloudgen.uniform_cloud(5000, seed=5)
    flat[:, 2] = 0.25
    np.testing.assert_array_equal(gpu_fps(rf, flat, 1000, 0), oracle.fps(flat, 1000, 0))
    line = np.zeros((4000, 3), np.float32)
    line[:, 0] = np.linspace(-3, 5, 4000, dtype=np.float32)
    np.testing.assert_array_equal(gpu_fps(rf, line, 4000, 0), oracle.fps(line, 4000, 0))
    wide = cloudgen.uniform_cloud(4000, seed=6) * np.float32(1e15)
    np.testing.assert_array_equal(gpu_fps(rf, wide, 800, 0), oracle.fps(wide, 800, 0))
    tiny = cloudgen.uniform_cloud(4000, seed=7) * np.float32(1e-20)
    np.testing.assert_array_equal(gpu_fps(rf, tiny, 800, 0), oracle.fps(tiny, 800, 0))


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_plain_variants(rf, variant):
    for pts, m, start in ((cloudgen.uniform_cloud(4096, seed=0), 1024, 0),
                          (cloudgen.room_cloud(50001, seed=9), 2000, 7)):
        ref = oracle.fps(pts, m, start, threads=0)
        got = rf.plain_fps(dev(pts), m, start, variant=variant).cpu().numpy()
        np.testing.assert_array_equal(got, ref)


def _ragged(sizes, seed):
    clouds = []
    for b, n in enumerate(sizes):
        pts = cloudgen.room_cloud(n, seed=seed + b) if b % 2 == 0 else cloudgen.lidar_cloud(n, seed=seed + b)
        clouds.append(pts)
    return clouds


@pytest.mark.parametrize("opts", [None, {"cluster": 2}, {"cluster": 4, "n_vox": 12}])
def test_batched_matches_per_cloud_oracle(rf, opts):
    sizes = [1, 7, 3000, 12345, 800, 20000, 64, 5000]
    clouds = _ragged(sizes, 100)
    ms = [max(1, n // 4) for n in sizes]
    starts = [n // 3 for n in sizes]
    cat = dev(np.concatenate(clouds))
    out, ooff = rf.fps_batched(cat, sizes, ms, starts, opts=opts)
    out = out.cpu().numpy()
    for b, pts in enumerate(clouds):
        ref = oracle.fps(pts, ms[b], starts[b], threads=0)
        np.testing.assert_array_equal(out[ooff[b]:ooff[b + 1]], ref, err_msg=f"cloud {b}")


@pytest.mark.parametrize("variant", [0, 1])
def test_plain_batched(rf, variant):
    sizes = [5, 3000, 12345, 800, 2048]
    clouds = _ragged(sizes, 200)
    ms = [max(1, n // 4) for n in sizes]
    out, ooff = rf.plain_fps_batched(dev(np.concatenate(clouds)), sizes, ms, variant=variant)
    out = out.cpu().numpy()
    for b, pts in enumerate(clouds):
        np.testing.assert_array_equal(out[ooff[b]:ooff[b + 1]], oracle.fps(pts, ms[b], 0, threads=0))


def test_host_buffers(rf):
    pts = cloudgen.room_cloud(30000, seed=21)
    ref = oracle.fps(pts, 7000, 11, threads=0)
    np.testing.assert_array_equal(rf.fps_host(pts, 7000, 11), ref)


def test_index_reuse(rf):
    pts = cloudgen.lidar_cloud(40000, seed=22)
    ix = rf.Index(dev(pts))
    for m, start in ((5000, 0), (100, 39999), (10000, 1234), (5000, 0)):
        got = ix.sample(m, start).cpu().numpy()
        np.testing.assert_array_equal(got, oracle.fps(pts, m, start, threads=0))
    assert ix.nbytes > 0
    ix.free()


def test_index_matches_oracle_voxel_grid(rf):
    """The device index agrees with the oracle's voxel grid (Sec. 3.2) bit for bit."""
    pts = cloudgen.room_cloud(25000, seed=23)
    for n_vox, chunk in ((16, 256), (33, 32)):
        ix = rf.Index(dev(pts), opts={"n_vox": n_vox, "chunk": chunk})
        e = ix.export()
        grid, vid = oracle.voxelize(pts, n_vox)
        assert e["n_vox"] == n_vox
        assert np.array_equal(e["grid_min"], grid["min"]) and e["L"] == grid["L"]
        orig = e["sorted_orig"]
        assert sorted(orig.tolist()) == list(range(len(pts)))
        # every record: one voxel, consecutive sorted positions, <= chunk points
        pos_vid = np.empty(len(pts), np.uint32)
        for r in range(len(e["first"])):
            a, c = int(e["first"][r]), int(e["count"][r])
            assert 1 <= c <= chunk
            pos_vid[a:a + c] = e["voxel_id"][r]
            members = orig[a:a + c]
            assert np.all(vid[members] == e["voxel_id"][r])
            # centre = p_min + (v + 1/2) L in FP32, radius covers every member exactly
            v = int(e["voxel_id"][r])
            vv = np.array([v % n_vox, (v // n_vox) % n_vox, v // (n_vox * n_vox)], np.float32)
            cen = grid["min"] + (vv + np.float32(0.5)) * grid["L"]
            assert np.array_equal(e["sphere"][r, :3], cen.astype(np.float32))
            d = np.sqrt(((pts[members].astype(np.float64) - cen.astype(np.float64)) ** 2).sum(1)).max()
            assert e["sphere"][r, 3] >= d and e["sphere"][r, 3] <= d * (1 + 2 ** -18) + 2 ** -49
        assert np.array_equal(pos_vid, vid[orig])
        # sorted by (Morton code of the voxel, original index): stable grouping in Z order
        vv = vid[orig].astype(np.int64)
        vx, vy, vz = vv % n_vox, (vv // n_vox) % n_vox, vv // (n_vox * n_vox)
        code = np.zeros_like(vv)
        for bit in range(10):
            code |= ((vx >> bit) & 1) << (3 * bit) | ((vy >> bit) & 1) << (3 * bit + 1) | ((vz >> bit) & 1) << (3 * bit + 2)
        key = code * len(pts) + orig
        assert np.all(np.diff(key) > 0)
        ix.free()


def test_nonfinite_is_reported(rf):
    pts = cloudgen.uniform_cloud(1000, seed=3)
    pts[500, 1] = np.nan
    with pytest.raises(rf.RfpsError) as e:
        rf.fps(dev(pts), 10, 0, check=True)
    assert e.value.status == 2
    pts[500, 1] = np.inf
    with pytest.raises(rf.RfpsError):
        rf.fps_host(pts, 10, 0)
    # the workspace is usable again after the error
    good = cloudgen.uniform_cloud(1000, seed=3)
    np.testing.assert_array_equal(gpu_fps(rf, good, 100, 0), oracle.fps(good, 100, 0))


def test_counters(rf):
    """Pruning and skipping do real work on a room-like cloud (the Tab. ablation statistic)."""
    pts = cloudgen.room_cloud(50000, seed=31)
    ws = torch.empty(rf.workspace_size(50000, {"counters": 1}), dtype=torch.uint8, device="cuda")
    out = rf.fps(dev(pts), 5000, 0, opts={"counters": 1}, workspace=ws)
    c = rf.counters(ws)
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.fps(pts, 5000, 0, threads=0))
    assert c["iterations"] == 4999
    assert c["voxels_pruned"] > 0.8 * c["voxel_tests"]
    assert c["points_skipped"] > 0 and c["points_updated"] > 50000
    assert c["points_visited"] < 0.2 * 50000 * 4999



@pytest.mark.parametrize("opts,n,shortcut", [({"cluster": 16, "threads": 128, "chunk": 64}, 40000, True),
                                              ({"cluster": 4, "threads": 256}, 40000, True),
                                              ({"cluster": 1, "threads": 256}, 40000, True),
                                              ({"cluster": 1, "threads": 512}, 4000, True),
                                              ({"cluster": 1, "threads": 256, "chunk": 32, "n_vox": 40}, 60000, True),
                                              ({"cluster": 1, "threads": 256, "chunk": 32, "n_vox": 40, "prune": 0},
                                               60000, True)],
                         ids=["c16_t128", "c4_t256", "one_cta", "register_records", "hierarchical",
                              "hierarchical_no_prune"])
def test_runner_up_shortcut_rounds(rf, opts, n, shortcut):
    """Every path (records in shared memory on clusters or one CTA, the register-record kernel, the
    hierarchical path with records in global memory: about one point per cell of a uniform cloud)
    selects the runner-up as the next sample too when the new sample leaves it unchanged: fewer
    selection rounds than samples, the oracle's indices all the same."""
    pts = cloudgen.uniform_cloud(n, seed=33) if "n_vox" in opts else cloudgen.room_cloud(n, seed=33)
    m = n * 3 // 20
    o = dict(opts, counters=1)
    ws = torch.empty(rf.workspace_size(n, o), dtype=torch.uint8, device="cuda")
    out = rf.fps(dev(pts), m, 5, opts=o, workspace=ws)
    c = rf.counters(ws)
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.fps(pts, m, 5, threads=0))
    assert c["iterations"] == m - 1
    if shortcut:
        assert (m - 1) / 2 <= c["rounds"] < 0.75 * (m - 1), c
    else:
        assert c["rounds"] == m - 1
    assert c["prune_violations"] == 0 and c["skip_violations"] == 0

SHADOW_CASES = [
    ("room_20k_c16_t128", lambda: cloudgen.room_cloud(20000, seed=81), 3000, {"cluster": 16, "threads": 128}),
    ("room_20k_c1", lambda: cloudgen.room_cloud(20000, seed=82), 3000, {"cluster": 1}),
    ("lidar_30k_c4", lambda: cloudgen.lidar_cloud(30000, seed=83), 3000, {"cluster": 4, "threads": 512}),
    ("lattice_ties_c8", lambda: _lattice(20, 20, 20), 2000, {"cluster": 8}),
    ("wide_scale_c16", lambda: cloudgen.uniform_cloud(8000, seed=84) * np.float32(3e12), 1500, {"cluster": 16}),
    ("tiny_scale_c2", lambda: cloudgen.uniform_cloud(8000, seed=85) * np.float32(1e-15), 1500, {"cluster": 2}),
    ("duplicates_c16", lambda: cloudgen.uniform_cloud(500, seed=86)[np.random.default_rng(87).integers(0, 500, 6000)],
     1000, {"cluster": 16}),
    ("hierarchical_c1", lambda: cloudgen.uniform_cloud(60000, seed=88), 300, {"cluster": 1, "chunk": 32, "n_vox": 40}),
]


@pytest.mark.parametrize("name,make,m,opts", SHADOW_CASES, ids=[c[0] for c in SHADOW_CASES])
def test_shadow_checks_find_no_unsafe_prune_or_skip(rf, name, make, m, opts):
    """Counting runs also check every pruned record's points and every skipped point against the new
    sample: no stored distance may be due for a strict decrease there, so the FP32 radius bound
    (Eq. radius_pruning_condition) and the coordinate skip (Eq. point_skip_condition) lose nothing."""
    pts = make().astype(np.float32)
    o = dict(opts, counters=1)
    ws = torch.empty(rf.workspace_size(pts.shape[0], o), dtype=torch.uint8, device="cuda")
    out = rf.fps(dev(pts), m, 0, opts=o, workspace=ws)
    c = rf.counters(ws)
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.fps(pts, m, 0, threads=0))
    assert c["voxels_pruned"] > 0 and c["points_skipped"] > 0
    assert c["prune_violations"] == 0 and c["skip_violations"] == 0, c


def test_launch_counter_moves(rf):
    before = rf.launch_count()
    gpu_fps(rf, cloudgen.uniform_cloud(500, seed=1), 50)
    assert rf.launch_count() > before


@pytest.mark.parametrize("opts", [None, {"cluster": 1, "chunk": 32}, {"cluster": 4}, {"cluster": 1, "n_vox": 40, "chunk": 32}])
def test_incremental_sampling_continues_the_sequence(rf, opts):
    """sample(m1) then sample_more(m2), sample_more(m3) equals one FPS run of m1 + m2 + m3 samples."""
    pts = cloudgen.room_cloud(40000, seed=51)
    ref = oracle.fps(pts, 9000, 3, threads=0)
    ix = rf.Index(dev(pts), opts=opts)
    a = ix.sample(2000, 3).cpu().numpy()
    b = ix.sample_more(1).cpu().numpy()
    c = ix.sample_more(6999).cpu().numpy()
    np.testing.assert_array_equal(np.concatenate([a, b, c]), ref)
    # a new sequence on the same index
    np.testing.assert_array_equal(ix.sample(500, 0).cpu().numpy(), oracle.fps(pts, 500, 0, threads=0))
    np.testing.assert_array_equal(ix.sample_more(100).cpu().numpy(), oracle.fps(pts, 600, 0, threads=0)[500:])
    with pytest.raises(rf.RfpsError):
        ix.sample_more(40000)
    ix.free()


def test_incremental_sampling_with_records_in_global_memory(rf):
    """Resume where most voxel records live in global memory (one CTA, fine voxels, tiny records)."""
    pts = cloudgen.uniform_cloud(60000, seed=52)
    ref = oracle.fps(pts, 3000, 0, threads=0)
    ix = rf.Index(dev(pts), opts={"cluster": 1, "n_vox": 40, "chunk": 32})
    got = [ix.sample(1000, 0).cpu().numpy(), ix.sample_more(1500).cpu().numpy(), ix.sample_more(500).cpu().numpy()]
    np.testing.assert_array_equal(np.concatenate(got), ref)
    ix.free()


@pytest.mark.parametrize("name,opts", [
    ("lidar_200k_c1", {"cluster": 1}),
    ("lidar_200k_c2_nv64", {"cluster": 2, "n_vox": 64}),
    ("room_150k_c1_chunk32", {"cluster": 1, "chunk": 32, "n_vox": 48}),
    ("uniform_120k_c1", {"cluster": 1, "n_vox": 64, "chunk": 64, "threads": 512}),
])
def test_hierarchical_path_many_records(rf, name, opts):
    """Clouds whose records exceed one CTA's shared memory: super-record pruning, records in global memory."""
    if name.startswith("lidar"):
        pts = cloudgen.lidar_cloud(200000, seed=61)
    elif name.startswith("room"):
        pts = cloudgen.room_cloud(150000, seed=62)
    else:
        pts = cloudgen.uniform_cloud(120000, seed=63)
    m = 6000
    ref = oracle.fps(pts, m, 11, threads=0)
    np.testing.assert_array_equal(gpu_fps(rf, pts, m, 11, **opts), ref)


def _lattice(nx, ny, nz):
    g = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    return np.stack([a.ravel() for a in g], 1).astype(np.float32)


@pytest.mark.parametrize("opts", [
    dict(cluster=2, threads=256), dict(cluster=4, threads=512), dict(cluster=8, threads=256),
    dict(cluster=16, threads=256), dict(cluster=16, threads=512), dict(cluster=16, threads=128),
], ids=lambda o: "c%d_t%d" % (o["cluster"], o["threads"]))
def test_exact_ties_across_cluster_exchange(rf, opts):
    """Equal squared distances in different warps and CTAs: the smallest point index must win (Sec. 3.1)."""
    grid = _lattice(16, 16, 16)
    np.testing.assert_array_equal(gpu_fps(rf, grid, 2000, 7, **opts), oracle.fps(grid, 2000, 7))
    base = cloudgen.uniform_cloud(3000, seed=71)
    dup = base[np.random.default_rng(72).permutation(np.repeat(np.arange(3000), 3))]
    # past 3000 samples every remaining candidate is at distance 0: each round is a tie
    np.testing.assert_array_equal(gpu_fps(rf, dup, 4000, 0, **opts), oracle.fps(dup, 4000, 0))
    same = np.tile(np.array([[0.5, 0.25, -3.0]], np.float32), (1000, 1))
    np.testing.assert_array_equal(gpu_fps(rf, same, 50, 999, **opts), oracle.fps(same, 50, 999))


def test_exact_ties_hierarchical_cluster(rf):
    """Ties on the hierarchical path (records in global memory) inside a 2-CTA cluster."""
    grid = _lattice(64, 64, 48)
    ref = oracle.fps(grid, 3000, 5, threads=0)
    np.testing.assert_array_equal(gpu_fps(rf, grid, 3000, 5, cluster=2, n_vox=64, chunk=32), ref)


D2_CASES = [
    ("room_20k_c16_t128", lambda: cloudgen.room_cloud(20000, seed=91), {"cluster": 16, "threads": 128}),
    ("lidar_30k_c4", lambda: cloudgen.lidar_cloud(30000, seed=92), {"cluster": 4}),
    ("lattice_ties_c8", lambda: _lattice(16, 16, 16), {"cluster": 8}),
    ("partly_resident_c1", lambda: cloudgen.lidar_cloud(40000, seed=93), {"cluster": 1, "threads": 512}),
    ("hierarchical_c1", lambda: cloudgen.uniform_cloud(60000, seed=94), {"cluster": 1, "chunk": 32, "n_vox": 40}),
]


@pytest.mark.parametrize("name,make,opts", D2_CASES, ids=[c[0] for c in D2_CASES])
def test_distance_state_matches_oracle_bit_for_bit(rf, name, make, opts):
    """Alg. 1's D after M samples: every point's stored FP32 squared distance equals the oracle's,
    bit for bit (pruned and skipped points included, since pruning and skipping are exact), after
    rfps_index_sample and again after rfps_index_sample_more."""
    pts = make().astype(np.float32)
    n = pts.shape[0]
    m1, m2 = n // 20, n // 40
    ix = rf.Index(dev(pts), opts=opts)
    idx1 = ix.sample(m1, 3).cpu().numpy()
    d1 = ix.distances().cpu().numpy()
    ref1, rd1 = oracle.fps(pts, m1, 3, threads=0, return_d2=True)
    np.testing.assert_array_equal(idx1, ref1)
    np.testing.assert_array_equal(d1.view(np.uint32), np.asarray(rd1, np.float32).view(np.uint32))
    idx2 = ix.sample_more(m2).cpu().numpy()
    d2 = ix.distances().cpu().numpy()
    ref2, rd2 = oracle.fps(pts, m1 + m2, 3, threads=0, return_d2=True)
    np.testing.assert_array_equal(idx2, ref2[m1:])
    np.testing.assert_array_equal(d2.view(np.uint32), np.asarray(rd2, np.float32).view(np.uint32))
    ix.free()


def _fuzz_cloud(rng, kind, n):
    if kind == "uniform":
        return cloudgen.uniform_cloud(n, seed=int(rng.integers(1 << 30)))
    if kind == "room":
        return cloudgen.room_cloud(n, seed=int(rng.integers(1 << 30)))
    if kind == "lidar":   # random subsets of one scan (generating a scan per seed is slow)
        return cloudgen.lidar_cloud(n, seed=int(rng.integers(1 << 30)), scan_seed=0)
    if kind == "lattice":
        side = max(1, int(round(n ** (1 / 3))))
        g = _lattice(side, side, max(1, n // (side * side)))
        return g[:n] if g.shape[0] >= n else np.concatenate([g, g[: n - g.shape[0]]])
    if kind == "duplicates":
        base = cloudgen.uniform_cloud(max(1, n // 7), seed=int(rng.integers(1 << 30)))
        return base[rng.integers(0, base.shape[0], n)]
    flat = cloudgen.uniform_cloud(n, seed=int(rng.integers(1 << 30)))
    flat[:, int(rng.integers(3))] = np.float32(rng.uniform(-5, 5))
    return flat


def _fuzz_opts(rng):
    o = {"cluster": int(rng.choice([1, 2, 4, 8, 16])), "threads": int(rng.choice([128, 256, 512])),
         "chunk": int(rng.choice([32, 64, 128, 256, 1024, 4096]))}
    if rng.random() < 0.5:
        o["n_vox"] = int(rng.integers(1, 97))
    if rng.random() < 0.2:
        o["prune"] = 0
    if rng.random() < 0.2:
        o["skip"] = 0
    if rng.random() < 0.2:
        o["radius_mode"] = 1
    return o


KINDS = ["uniform", "room", "lidar", "lattice", "duplicates", "flat"]


@pytest.mark.parametrize("seed", range(24))
def test_fuzz_single_cloud(rf, seed):
    """Seeded random cloud kind, size, M, start and option set: indices equal the oracle's."""
    rng = np.random.default_rng(1000 + seed)
    kind = KINDS[seed % len(KINDS)]
    n = int(np.exp(rng.uniform(0, np.log(40000))))
    pts = _fuzz_cloud(rng, kind, n).astype(np.float32)
    n = pts.shape[0]
    m = int(rng.integers(1, min(n, 3000) + 1))
    start = int(rng.integers(0, n))
    o = _fuzz_opts(rng)
    np.testing.assert_array_equal(gpu_fps(rf, pts, m, start, **o), oracle.fps(pts, m, start, threads=0),
                                  err_msg=f"{kind} n={n} m={m} start={start} {o}")


def _tie_cloud(rng, kind, n):
    """Clouds full of exactly equal squared distances: small-integer coordinates, mirror images, a
    ring of equally spaced points around equal blobs, a coarse quantised grid."""
    if kind == "integers":
        return rng.integers(0, 6, size=(n, 3)).astype(np.float32)
    if kind == "mirrored":
        half = cloudgen.uniform_cloud(max(1, n // 2), seed=int(rng.integers(1 << 30)))
        return np.concatenate([half, -half])[:n]
    if kind == "ring":
        k = max(3, n // 40)
        ang = 2 * np.pi * np.arange(k) / k
        centres = np.stack([np.cos(ang), np.sin(ang), np.zeros(k)], 1) * 64
        blob = rng.integers(-2, 3, size=(max(1, n // k), 3))
        return (centres[:, None, :] + blob[None, :, :]).reshape(-1, 3)[:n].astype(np.float32)
    return np.round(cloudgen.room_cloud(n, seed=int(rng.integers(1 << 30))) * 4) / 4   # quantised


@pytest.mark.parametrize("seed", range(24))
def test_fuzz_ties(rf, seed):
    """Exact ties everywhere (the case the runner-up shortcut's strict bound and d2 > 0 rule guard):
    seeded tie-heavy clouds under random options, the register-record path included."""
    rng = np.random.default_rng(3000 + seed)
    kind = ["integers", "mirrored", "ring", "quantised"][seed % 4]
    n = int(np.exp(rng.uniform(np.log(50), np.log(30000))))
    pts = np.ascontiguousarray(_tie_cloud(rng, kind, n), dtype=np.float32)
    n = pts.shape[0]
    m = int(rng.integers(1, min(n, 2500) + 1))
    start = int(rng.integers(0, n))
    o = {"cluster": 1, "threads": 512} if seed % 3 == 0 else _fuzz_opts(rng)
    np.testing.assert_array_equal(gpu_fps(rf, pts, m, start, **o), oracle.fps(pts, m, start, threads=0),
                                  err_msg=f"{kind} n={n} m={m} start={start} {o}")


@pytest.mark.parametrize("seed", range(6))
def test_fuzz_batched(rf, seed):
    """Seeded random ragged batches (kinds, sizes, M, starts) under a random option set."""
    rng = np.random.default_rng(2000 + seed)
    b = int(rng.integers(1, 12))
    clouds = [_fuzz_cloud(rng, KINDS[int(rng.integers(len(KINDS)))], int(np.exp(rng.uniform(0, np.log(20000)))))
              .astype(np.float32) for _ in range(b)]
    sizes = [c.shape[0] for c in clouds]
    ms = [int(rng.integers(1, min(n, 1500) + 1)) for n in sizes]
    starts = [int(rng.integers(0, n)) for n in sizes]
    o = _fuzz_opts(rng)
    out, ooff = rf.fps_batched(dev(np.concatenate(clouds)), sizes, ms, starts, opts=o)
    out = out.cpu().numpy()
    for i, c in enumerate(clouds):
        np.testing.assert_array_equal(out[ooff[i]:ooff[i + 1]], oracle.fps(c, ms[i], starts[i], threads=0),
                                      err_msg=f"cloud {i} n={sizes[i]} {o}")


def test_batched_rejects_bad_device_metadata(rf):
    """Per-cloud arrays are checked on the device (Alg. 2 preprocessing takes them as given): a
    sample count above the cloud size, a start outside it, or offsets that do not cover the points
    end the call with RFPS_EINVAL in the status word, and the workspace then serves a valid batch."""
    sizes = [500, 800, 300]
    clouds = [cloudgen.uniform_cloud(n, seed=40 + i) for i, n in enumerate(sizes)]
    cat = dev(np.concatenate(clouds))
    ws = torch.empty(rf.batch_workspace_size(cat.shape[0], 3, max(sizes)), dtype=torch.uint8, device="cuda")
    for ms, starts in (([10, 900, 5], [0, 0, 0]), ([10, 20, 5], [0, 800, 0]), ([10, 20, 5], [0, -1, 0])):
        meta = rf._lib._batch_meta(sizes, ms, starts, cat.device)
        rf.fps_batched(cat, sizes, ms, starts, workspace=ws, meta=meta)
        assert rf.status(ws) == 1, (ms, starts)
    d_off, d_ooff, d_st, off, ooff, max_n = rf._lib._batch_meta(sizes, [10, 20, 5], [0, 0, 0], cat.device)
    short = d_off.clone()
    short[-1] = short[-1] - 1                      # offsets end before the last point
    rf.fps_batched(cat, sizes, [10, 20, 5], [0, 0, 0], workspace=ws, meta=(short, d_ooff, d_st, off, ooff, max_n))
    assert rf.status(ws) == 1
    ms = [100, 200, 50]
    out, oo = rf.fps_batched(cat, sizes, ms, [0, 0, 0], workspace=ws)
    assert rf.status(ws) == 0
    out = out.cpu().numpy()
    for b, c in enumerate(clouds):
        np.testing.assert_array_equal(out[oo[b]:oo[b + 1]], oracle.fps(c, ms[b], 0))


@pytest.mark.parametrize("name,make,opts", [
    ("uniform_7_c1", lambda: cloudgen.uniform_cloud(7, seed=3), {"cluster": 1}),
    ("uniform_64_c16", lambda: cloudgen.uniform_cloud(64, seed=4), {"cluster": 16, "threads": 128}),
    ("room_64_c4", lambda: cloudgen.room_cloud(64, seed=5), {"cluster": 4}),
    ("lattice_ties_c2", lambda: _lattice(4, 4, 4), {"cluster": 2, "chunk": 32, "n_vox": 3}),
    ("duplicates_c8", lambda: cloudgen.uniform_cloud(9, seed=6)[np.arange(48) % 9], {"cluster": 8}),
])
def test_distance_state_every_iteration_small(rf, name, make, opts):
    """Small clouds stepped one sample at a time (rfps_index_sample_more(1)): after every iteration the
    whole distance array D equals the oracle's bit for bit, and so does the new index."""
    pts = make().astype(np.float32)
    n = pts.shape[0]
    start = n // 3
    ix = rf.Index(dev(pts), opts=opts)
    got = list(ix.sample(2, start).cpu().numpy())
    for m in range(2, n + 1):
        if m > 2:
            got.append(int(ix.sample_more(1).cpu().numpy()[0]))
        ref, rd = oracle.fps(pts, m, start, threads=0, return_d2=True)
        np.testing.assert_array_equal(np.array(got), ref, err_msg=f"m={m}")
        d = ix.distances().cpu().numpy()
        np.testing.assert_array_equal(d.view(np.uint32), np.asarray(rd, np.float32).view(np.uint32), err_msg=f"m={m}")
    ix.free()


@pytest.mark.parametrize("opts", [{"cluster": 4, "threads": 256}, {"cluster": 16, "threads": 128},
                                  {"cluster": 1, "threads": 512}], ids=["c4", "c16", "register_records"])
def test_runner_up_shortcut_at_the_sequence_ends(rf, opts):
    """The runner-up shortcut never takes a cloud's last sample, so short runs and every resume
    boundary of a kept index still give the oracle's sequence: M = 1 to 6, and pieces of one to
    five samples continued with sample_more."""
    n = 4000 if opts["cluster"] == 1 else 30000
    pts = cloudgen.room_cloud(n, seed=57)
    ref = oracle.fps(pts, 60, 11, threads=0)
    for m in range(1, 7):
        np.testing.assert_array_equal(gpu_fps(rf, pts, m, 11, **opts), ref[:m])
    ix = rf.Index(dev(pts), opts=opts)
    got = [ix.sample(3, 11).cpu().numpy()]
    for k in (1, 2, 3, 4, 5, 1, 2, 3, 4, 5, 1, 2, 3, 4, 5, 1):
        got.append(ix.sample_more(k).cpu().numpy())
    np.testing.assert_array_equal(np.concatenate(got), ref[:sum(len(g) for g in got)])
    ix.free()
