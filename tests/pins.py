"""Pins of the CPU oracle: checks against what the paper and the mathematics fix.

Each ``pin_*`` function takes a loaded oracle library (``oracle.load(path)``)
and raises AssertionError on the first disagreement.  ``test_oracle_pins.py``
runs them against the oracle; ``test_oracle_mutants.py`` runs them against
copies of the oracle with a planted mistake and requires that some pin fails.
"""

from __future__ import annotations

import json
import os

import numpy as np

import cloudgen
import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)["cases"]


def _cover2(points, out):
    """Squared coverage radius at each selection: min over earlier samples of d2."""
    p = np.asarray(points, dtype=np.float32)
    d = np.full(p.shape[0], np.inf, dtype=np.float32)
    cov = []
    for j in range(1, len(out)):
        d = np.minimum(d, oracle.sq_dist_np(p, p[out[j - 1]]))
        cov.append(float(d[out[j]]))
    return cov


def pin_golden_fps(lib):
    """Hand-worked examples (Alg. 1, Sec. 3.1) for plain FPS and every RadiusFPS switch."""
    for case in _golden("fps_hand_worked.json"):
        pts = np.array(case["points"], dtype=np.float32)
        if "points_bits" in case:
            pts = np.array(case["points_bits"], dtype=np.uint32).view(np.float32)
        exp = case["expected"]
        got = oracle.fps(pts, case["m"], case["start"], lib=lib)
        assert got.tolist() == exp, (case["name"], got.tolist(), exp)
        got_mt = oracle.fps(pts, case["m"], case["start"], threads=3, lib=lib)
        assert got_mt.tolist() == exp, (case["name"], "threads", got_mt.tolist())
        np.testing.assert_array_equal(np.array(_cover2(pts, exp), dtype=np.float32),
                                      np.array(case["cover2"], dtype=np.float32))
        for n_vox in (1, 2, 3, 8):
            for prune in (0, 1):
                for skip in (0, 1):
                    for rm in (0, 1):
                        g, _ = oracle.radiusfps(pts, case["m"], case["start"], n_vox, prune, skip, rm,
                                                lib=lib)
                        assert g.tolist() == exp, (case["name"], n_vox, prune, skip, rm, g.tolist())


def pin_bruteforce(lib):
    """Incremental FPS equals the from-scratch argmax-min definition on tiny clouds."""
    rng = np.random.default_rng(12345)
    for trial in range(60):
        n = int(rng.integers(1, 48))
        kind = trial % 4
        if kind == 0:
            pts = rng.random((n, 3), dtype=np.float32)
        elif kind == 1:    # small integer grid: many exact ties
            pts = rng.integers(-3, 4, size=(n, 3)).astype(np.float32)
        elif kind == 2:    # duplicates
            base = rng.random((max(1, n // 3), 3), dtype=np.float32)
            pts = base[rng.integers(0, base.shape[0], size=n)]
        else:              # mixed scales, negative coordinates
            pts = (rng.standard_normal((n, 3)) * 10.0 ** rng.integers(-3, 4, size=(n, 1))).astype(np.float32)
        m = int(rng.integers(1, n + 1))
        start = int(rng.integers(0, n))
        exp = oracle.fps_bruteforce(pts, m, start)
        got = oracle.fps(pts, m, start, lib=lib)
        assert np.array_equal(got, exp), (trial, n, m, start, got, exp)


def pin_invariants(lib):
    """Invariants of FPS on moderate clouds: distinct samples, non-increasing coverage,
    stored distances equal the min over the samples, M = N gives a permutation."""
    for name, pts in (("uniform", cloudgen.uniform_cloud(3000, seed=3)),
                      ("room", cloudgen.room_cloud(3000, seed=4))):
        m = 700
        out, d2 = oracle.fps(pts, m, 5, return_d2=True, lib=lib)
        assert out[0] == 5
        assert len(set(out.tolist())) == m, name
        cov = np.array(_cover2(pts, out.tolist()))
        assert np.all(np.diff(cov) <= 0), name
        # d2 after the last update = min over samples s_0 .. s_{m-2}
        ref = np.full(pts.shape[0], np.inf, dtype=np.float32)
        for s in out[:-1]:
            ref = np.minimum(ref, oracle.sq_dist_np(pts, pts[s]))
        assert np.array_equal(d2, ref), name
        # the last sample is the argmax of that state, first index on ties
        assert out[-1] == int(np.argmax(ref)), name
    pts = cloudgen.uniform_cloud(257, seed=9)
    out = oracle.fps(pts, 257, 0, lib=lib)
    assert sorted(out.tolist()) == list(range(257))


def pin_closed_form(lib):
    """Points 0, 1, 2, 4, ..., 2^(n-2) on a line, start 0: FPS takes them in
    descending order (each 2^k is at distance 2^k from both its neighbours
    among the samples).  Also along y and z, and mirrored."""
    for axis in range(3):
        for sign in (1.0, -1.0):
            n = 20
            xs = [0.0] + [2.0 ** k for k in range(n - 1)]
            pts = np.zeros((n, 3), dtype=np.float32)
            pts[:, axis] = sign * np.array(xs, dtype=np.float32)
            got = oracle.fps(pts, n, 0, lib=lib).tolist()
            assert got == [0] + list(range(n - 1, 0, -1)), (axis, sign, got)


def pin_radiusfps_identity(lib):
    """CPU RadiusFPS with every prune/skip switch returns the plain FPS indices
    (the exactness claim of Sec. 3.4: Eq. global_equivalent_selection,
    radius_pruning_correctness and the point-skip argument)."""
    clouds = [
        ("uniform", cloudgen.uniform_cloud(4000, seed=1), 1000, 0),
        ("room", cloudgen.room_cloud(6000, seed=2), 1500, 17),
        ("lidar", cloudgen.lidar_cloud(6000, seed=3), 1500, 0),
        ("grid_ties", np.array(np.meshgrid(*[np.arange(12)] * 3), dtype=np.float32).reshape(3, -1).T.copy(),
         600, 0),
    ]
    for name, pts, m, start in clouds:
        ref = oracle.fps(pts, m, start, lib=lib)
        for n_vox in (4, 11, 24):
            for prune, skip in ((1, 1), (1, 0), (0, 1)):
                got, st = oracle.radiusfps(pts, m, start, n_vox, prune, skip, 0, lib=lib)
                assert np.array_equal(got, ref), (name, n_vox, prune, skip)
        got, st = oracle.radiusfps(pts, m, start, 16, 1, 1, 1, lib=lib)
        assert np.array_equal(got, ref), (name, "paper radius")
        assert st["voxels_pruned"] > 0, name


def pin_voxelize(lib):
    """Voxel grid (Sec. 3.2): hand-worked cells, and on generated clouds every
    point lies in its cell's cube up to one rounding, ids in range, L as defined."""
    for case in _golden("voxel_grid_hand_worked.json"):
        pts = np.array(case["points"], dtype=np.float32)
        grid, vid = oracle.voxelize(pts, case["n_vox"], lib=lib)
        assert grid["L"] == np.float32(case["L"]), (case["name"], grid["L"])
        assert vid.tolist() == case["expected_vid"], (case["name"], vid.tolist())
    for n_vox in (1, 7, 32):
        pts = cloudgen.room_cloud(5000, seed=n_vox)
        grid, vid = oracle.voxelize(pts, n_vox, lib=lib)
        assert np.array_equal(grid["min"], pts.min(0)) and np.array_equal(grid["max"], pts.max(0))
        e = float((pts.max(0).astype(np.float64) - pts.min(0)).max())
        assert abs(float(grid["L"]) - (1 + 2 ** -10) * e / n_vox) <= 1e-6 * e
        v = np.stack([vid % n_vox, (vid // n_vox) % n_vox, vid // (n_vox * n_vox)], axis=1)
        assert vid.max() < n_vox ** 3
        rel = (pts.astype(np.float64) - grid["min"].astype(np.float64)) / float(grid["L"])
        assert np.all(rel >= v - 1e-5) and np.all(rel <= v + 1 + 1e-5)
