"""FP64 information report -- TEST INFRASTRUCTURE (calls only the oracle).

For each workload, runs the FP32 squared-distance oracle (the library's
canonical reading, C1/C2) and the FP64 square-root-domain oracle (the
real-number reading of Alg. 1) from the same start, and reports:

* the first step at which the two index sequences differ and the fraction
  of positions that differ (information only: once one index differs, the
  rest of the sequence follows a different path);
* the largest relative difference between the two runs' coverage radii at
  the same step (the distance of each newly selected point to the earlier
  samples), a measure of how much the sampling quality differs.

Usage: python oracle/f64_report.py [workload ...] [--m M]
"""

from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import cloudgen  # noqa: E402
import oracle  # noqa: E402


def report(points: np.ndarray, m: int, start: int = 0) -> dict:
    out32, d2 = oracle.fps(points, m, start, threads=0, return_d2=True)
    out64, cov64 = oracle.fps_f64(points, m, start)
    # FP32 run's coverage radius at each step, from a replay of its own selections in double
    p = points.astype(np.float64)
    d = np.full(p.shape[0], np.inf)
    cov32 = [np.inf]
    for j in range(1, m):
        s = p[out32[j - 1]]
        d = np.minimum(d, np.sqrt(((p - s) ** 2).sum(1)))
        cov32.append(d[out32[j]])
    cov32 = np.array(cov32)
    diff = np.nonzero(out32 != out64)[0]
    rel = np.abs(cov32[1:] - cov64[1:]) / np.maximum(cov64[1:], 1e-30)
    return {
        "n": int(points.shape[0]), "m": int(m),
        "first_divergence": int(diff[0]) if diff.size else None,
        "divergent_fraction": float(diff.size / m),
        "max_rel_coverage_diff": float(rel.max()) if rel.size else 0.0,
        "final_coverage_f32": float(cov32[-1]), "final_coverage_f64": float(cov64[-1]),
    }


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("workloads", nargs="*", default=["uniform4k", "room100k"])
    ap.add_argument("--m", type=int, default=0, help="samples (0: the workload's M)")
    args = ap.parse_args(argv)
    for w in args.workloads:
        clouds, desc = cloudgen.workload(w)
        c = clouds[0]
        r = report(c.points, args.m or c.m, c.start)
        r["workload"] = w
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
