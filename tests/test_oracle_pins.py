"""The CPU oracle against its pins (no GPU)."""

import json
import os

import numpy as np
import pytest

import cloudgen
import oracle
import pins


@pytest.fixture(scope="module")
def lib():
    return oracle.load()


def test_golden_fps(lib):
    pins.pin_golden_fps(lib)


def test_bruteforce(lib):
    pins.pin_bruteforce(lib)


def test_invariants(lib):
    pins.pin_invariants(lib)


def test_closed_form(lib):
    pins.pin_closed_form(lib)


def test_radiusfps_identity(lib):
    pins.pin_radiusfps_identity(lib)


def test_voxelize(lib):
    pins.pin_voxelize(lib)


def test_sqrt_domain_divergence():
    """Reading C1: an FP32 square-root-domain FPS would break the tie the other way."""
    case = [c for c in json.load(open(os.path.join(pins.GOLDEN, "fps_hand_worked.json")))["cases"]
            if c["name"] == "squared_vs_sqrt_domain"][0]
    pts = np.array(case["points_bits"], dtype=np.uint32).view(np.float32)
    d = np.full(3, np.inf, dtype=np.float32)
    sel = [0]
    for _ in range(2):
        d = np.minimum(d, np.sqrt(oracle.sq_dist_np(pts, pts[sel[-1]])))
        sel.append(int(np.argmax(d)))
    assert sel == case["sqrt_domain_fp32_expected"]
    assert oracle.fps(pts, 3, 0).tolist() == case["expected"]


def test_f64_info_oracle_on_exact_examples():
    """The FP64 square-root-domain oracle agrees on the hand-worked cases (all
    distances are exact there, so the readings coincide)."""
    for case in json.load(open(os.path.join(pins.GOLDEN, "fps_hand_worked.json")))["cases"]:
        pts = np.array(case["points"], dtype=np.float32)
        if "points_bits" in case:
            pts = np.array(case["points_bits"], dtype=np.uint32).view(np.float32)
        out, cov = oracle.fps_f64(pts, case["m"], case["start"])
        assert out.tolist() == case["expected"], case["name"]
        np.testing.assert_allclose(cov[1:] ** 2, case["cover2"], rtol=1e-6)


def test_threads_do_not_change_result():
    pts = cloudgen.room_cloud(20000, seed=5)
    a = oracle.fps(pts, 2000, 3, threads=1)
    b = oracle.fps(pts, 2000, 3, threads=4)
    c = oracle.fps(pts, 2000, 3, threads=0)
    assert np.array_equal(a, b) and np.array_equal(a, c)


def test_argument_errors():
    pts = cloudgen.uniform_cloud(10)
    with pytest.raises(oracle.OracleError):
        oracle.fps(pts, 11, 0)
    with pytest.raises(oracle.OracleError):
        oracle.fps(pts, 0, 0)
    with pytest.raises(oracle.OracleError):
        oracle.fps(pts, 3, 10)
    with pytest.raises(oracle.OracleError):
        oracle.fps(pts, 3, -1)
    bad = pts.copy()
    bad[4, 1] = np.nan
    with pytest.raises(oracle.OracleError, match="non-finite"):
        oracle.fps(bad, 3, 0)
    bad[4, 1] = np.inf
    with pytest.raises(oracle.OracleError, match="non-finite"):
        oracle.radiusfps(bad, 3, 0)


def test_single_point_and_m1():
    assert oracle.fps(np.zeros((1, 3), np.float32), 1, 0).tolist() == [0]
    assert oracle.fps(cloudgen.uniform_cloud(50), 1, 7).tolist() == [7]
    g, _ = oracle.radiusfps(np.zeros((1, 3), np.float32), 1, 0)
    assert g.tolist() == [0]


def test_radiusfps_prunes_and_skips():
    """Both filters do real work on a room-like cloud (the ablation of Tab. ablation)."""
    pts = cloudgen.room_cloud(20000, seed=8)
    ref = oracle.fps(pts, 5000, 0, threads=0)
    got, st = oracle.radiusfps(pts, 5000, 0, n_vox=24)
    assert np.array_equal(got, ref)
    assert st["voxels_pruned"] > 0.9 * st["voxel_tests"]
    assert st["points_skipped"] > 0
    assert st["points_updated"] < st["points_visited"]


def _canonical_d2(p, q):
    d = (p - q).astype(np.float32)
    return ((d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]).astype(np.float32)


@pytest.mark.parametrize("kind", ["room", "lidar", "lattice", "duplicates"])
def test_runner_up_shortcut_matches_the_oracle(kind):
    """The sampling kernel's runner-up shortcut, checked against the oracle's FPS sequence: whenever
    the runner-up r of the state that chose s_j (second-largest (d2, lowest index) key) has d2 > 0
    and its canonical squared distance to s_j is not below its d2, the oracle's next sample is r.
    Ties (the lattice) and zero distances (duplicates) are the cases the d2 > 0 and key rules
    exist for."""
    rng = np.random.default_rng(5)
    n, m = 3000, 700
    if kind == "room":
        pts = cloudgen.room_cloud(n, seed=61)
    elif kind == "lidar":
        pts = cloudgen.lidar_cloud(n, seed=62)
    elif kind == "lattice":
        g = np.arange(15, dtype=np.float32)
        pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)[:n].astype(np.float32)
    else:
        base = rng.random((n // 4, 3), dtype=np.float32)
        pts = np.repeat(base, 4, axis=0)
        m = n // 4 + 50   # past the distinct points: the remaining distances are 0
    pts = np.ascontiguousarray(pts, dtype=np.float32)
    seq = oracle.fps(pts, m, 0)
    d2 = np.full(pts.shape[0], np.inf, dtype=np.float32)
    idx = np.arange(pts.shape[0])
    fired = 0
    for j in range(1, m - 1):
        nd = _canonical_d2(pts, pts[seq[j - 1]])
        d2 = np.where(nd < d2, nd, d2)
        # (d2, lowest index) order: the oracle's next sample is the first key, r the second
        order = np.lexsort((idx, -d2.astype(np.float64)))
        t1, r = order[0], order[1]
        assert t1 == seq[j]
        if d2[r] > 0 and _canonical_d2(pts[r], pts[t1]) >= d2[r]:
            fired += 1
            assert seq[j + 1] == r, (j, r, seq[j + 1])
    # with four copies of every point the runner-up is a copy of the sample (distance 0): never taken
    assert fired > 0 if kind != "duplicates" else fired == 0
