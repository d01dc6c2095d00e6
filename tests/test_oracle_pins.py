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
