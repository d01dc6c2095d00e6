"""Small clouds on one CTA (N <= 4,096; options cluster 1, threads 512): each of 1,024 threads
holds up to 4 points as a record in registers (k_sample_regs; the library default for clouds this
small).  Element-by-element parity with the oracle over the sizes around the capacity (and past
it, where the same options run the shared-memory loop), exact ties, duplicates, prune / skip
switches, incremental sampling with the distance state, overflowing distances, the shadow checks
and ragged batches."""

import numpy as np
import pytest
import torch

import cloudgen
import oracle

pytestmark = pytest.mark.gpu

ONE_CTA = {"cluster": 1, "threads": 512}


@pytest.fixture(scope="module")
def rf():
    import paper_2606_06255_gb300 as rf
    return rf


def dev(p):
    return torch.from_numpy(np.ascontiguousarray(p, dtype=np.float32)).cuda()


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 511, 512, 513, 4095, 4096, 4097, 5003, 8191, 8192])
def test_sizes_around_the_register_capacities(rf, n):
    pts = cloudgen.uniform_cloud(n, seed=300 + n)
    m = max(1, n // 3)
    start = (7 * n) // 11
    got = rf.fps(dev(pts), m, start, opts=ONE_CTA, check=True).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.fps(pts, m, start))


@pytest.mark.parametrize("kind", ["room", "lidar", "lattice", "duplicates", "collinear"])
@pytest.mark.parametrize("opts", [{}, {"prune": 0}, {"skip": 0}, {"nvox_scale": 35}, {"n_vox": 2}, {"radius_mode": 1}],
                         ids=lambda o: str(o) or "default")
def test_structured_clouds_and_switches(rf, kind, opts):
    if kind == "room":
        pts = cloudgen.room_cloud(4000, seed=310)
    elif kind == "lidar":
        pts = cloudgen.lidar_cloud(3500, seed=311)
    elif kind == "lattice":          # equal distances everywhere: the smallest index must win
        g = np.meshgrid(np.arange(16), np.arange(16), np.arange(16), indexing="ij")
        pts = np.stack([a.ravel() for a in g], 1).astype(np.float32)
    elif kind == "duplicates":       # past 1,300 samples every candidate is at distance 0
        base = cloudgen.uniform_cloud(1300, seed=312)
        pts = base[np.random.default_rng(313).permutation(np.repeat(np.arange(1300), 3))]
    else:
        pts = np.zeros((3000, 3), np.float32)
        pts[:, 0] = np.arange(3000, dtype=np.float32) * 0.25
    assert pts.shape[0] <= 4096
    m = min(pts.shape[0], 2500)
    got = rf.fps(dev(pts), m, 5, opts=dict(ONE_CTA, **opts), check=True).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.fps(pts, m, 5, threads=0))


def test_uniform4k_workload(rf):
    (c,), _ = cloudgen.workload("uniform4k")
    assert rf.resolved_opts(4096)["threads"] == 512 and rf.resolved_opts(4096)["cluster"] == 1
    for opts in (None, ONE_CTA, dict(ONE_CTA, nvox_scale=35), dict(ONE_CTA, nvox_scale=140)):
        got = rf.fps(dev(c.points), c.m, c.start, opts=opts, check=True).cpu().numpy()
        np.testing.assert_array_equal(got, oracle.fps(c.points, c.m, c.start), err_msg=str(opts))


def test_incremental_sampling_and_distance_state(rf):
    """Pieces taken through the kept index equal one oracle run of the total M, and after each call
    the distance state (Alg. 1's D) equals the oracle's after the same number of samples, bit for bit."""
    pts = cloudgen.room_cloud(4000, seed=314)
    ref, d2 = oracle.fps(pts, 3000, 9, return_d2=True)
    _, d2_700 = oracle.fps(pts, 700, 9, return_d2=True)
    ix = rf.Index(dev(pts), opts=ONE_CTA)
    first = ix.sample(700, 9).cpu().numpy()
    np.testing.assert_array_equal(ix.distances().cpu().numpy().view(np.uint32), d2_700.view(np.uint32))
    got = [first, ix.sample_more(1300).cpu().numpy(), ix.sample_more(1000).cpu().numpy()]
    np.testing.assert_array_equal(np.concatenate(got), ref)
    np.testing.assert_array_equal(ix.distances().cpu().numpy().view(np.uint32), d2.view(np.uint32))
    ix.free()


def test_shadow_checks_and_counters(rf):
    pts = cloudgen.room_cloud(4000, seed=315)
    m = 1500
    opts = dict(ONE_CTA, counters=1)
    ws = torch.empty(rf.workspace_size(pts.shape[0], opts), dtype=torch.uint8, device="cuda")
    got = rf.fps(dev(pts), m, 0, opts=opts, workspace=ws).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.fps(pts, m, 0))
    c = rf.counters(ws)
    assert c["iterations"] == m - 1
    assert c["prune_violations"] == 0 and c["skip_violations"] == 0
    assert 0 < c["voxels_pruned"] < c["voxel_tests"]
    assert c["points_updated"] <= c["points_visited"] - c["points_skipped"]


def test_ragged_batch_of_small_clouds(rf):
    rng = np.random.default_rng(316)
    sizes = [int(x) for x in rng.integers(1, 4097, size=20)] + [4096, 1, 4095]
    clouds = [cloudgen.room_cloud(n, seed=400 + i) if i % 2 else cloudgen.uniform_cloud(n, seed=400 + i)
              for i, n in enumerate(sizes)]
    ms = [max(1, n // 4) for n in sizes]
    starts = [int(rng.integers(0, n)) for n in sizes]
    out, ooff = rf.fps_batched(dev(np.concatenate(clouds)), sizes, ms, starts, opts=ONE_CTA)
    out = out.cpu().numpy()
    for b, c in enumerate(clouds):
        np.testing.assert_array_equal(out[ooff[b]:ooff[b + 1]], oracle.fps(c, ms[b], starts[b]), err_msg=f"cloud {b}")


@pytest.mark.parametrize("opts", [ONE_CTA, {"cluster": 4, "threads": 128}], ids=["registers", "cluster4"])
def test_squared_distances_that_overflow(rf, opts):
    """Coordinates up to 4e19: many FP32 squared distances are +inf, so in the first iteration some
    distances stay +inf (not a strict decrease) and the record keys must still come from them."""
    pts = cloudgen.uniform_cloud(3000, seed=317) * np.float32(4e19)
    got = rf.fps(dev(pts), 1200, 3, opts=opts, check=True).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.fps(pts, 1200, 3))


def test_non_finite_coordinates_are_reported(rf):
    """The register path groups the points itself (no index build runs), so it also checks them:
    a NaN or an infinity anywhere gives RFPS_ENONFINITE, alone or in a batch, and the workspace then
    serves a clean call."""
    pts = cloudgen.room_cloud(3000, seed=318)
    for bad_value in (np.nan, np.inf, -np.inf):
        bad = pts.copy()
        bad[2999, 2] = bad_value
        ws = torch.empty(rf.workspace_size(3000, ONE_CTA), dtype=torch.uint8, device="cuda")
        rf.fps(dev(bad), 500, 0, opts=ONE_CTA, workspace=ws)
        assert rf.status(ws) == 2
        got = rf.fps(dev(pts), 500, 0, opts=ONE_CTA, workspace=ws).cpu().numpy()
        assert rf.status(ws) == 0
        np.testing.assert_array_equal(got, oracle.fps(pts, 500, 0))
    clouds = [cloudgen.uniform_cloud(1000 + 10 * i, seed=500 + i) for i in range(5)]
    clouds[3] = clouds[3].copy()
    clouds[3][7, 0] = np.nan
    sizes = [c.shape[0] for c in clouds]
    ws = torch.empty(rf.batch_workspace_size(sum(sizes), 5, max(sizes), ONE_CTA), dtype=torch.uint8, device="cuda")
    rf.fps_batched(dev(np.concatenate(clouds)), sizes, [100] * 5, opts=ONE_CTA, workspace=ws)
    assert rf.status(ws) == 2
