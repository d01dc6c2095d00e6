"""Benchmark of the RadiusFPS hot path on GB300: one JSON line on rank 0.

A step is one full pass of the path over one cloud: device-side voxel index
build (bounding box, binning, sort, records) plus the persistent sampling
kernel (initial update, then M - 1 select / prune / skip / update / resync
iterations).  Default workload: the accumulated rotating-LiDAR scan,
N = 1,124,730 points, M = 16,384 samples, start 0 (synthetic stand-in for the
paper's outdoor scenes, Sec. Computation Efficiency and Resource
Consumption), with the launch shape and voxel resolution picked by the
autotuner before the timed region.  The same line carries, as extra keys,
the room-like (N = 100,000, M = 25,000) and uniform (N = 4,096, M = 1,024)
single clouds, the 64-cloud ragged batch (clouds/s, graph-replayed batch
against per-cloud launches) and the Poisson serving run (p50 / p99 latency
at 200 clouds/s offered); --secondary none leaves them out.  Other headline
workloads: --workload uniform4k | room100k | batch64 | serving.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events
on the launching stream; between steps a 256 MiB buffer is written to flush
the 129 MB L2 (outside the events).  Barrier + synchronize on both sides of
the timed loop, max over ranks.  Multi-GPU: one process per GPU, each samples
its own cloud (clouds are independent units; no data-path collective).

The CPU baseline is the oracle as it stands, timed in a separate process
that holds no CUDA context, after the GPU work: plain FPS on every host core
(OpenMP) over the full workload, plain FPS on one thread over the first
samples of the workload, and the CPU RadiusFPS on one thread at the paper's
v = 32 (Sec. Hardware Acceleration and Parameter Sensitivity).

--impl reference times the CPU oracle (plain FPS, all host cores) on the
same workload and config instead (rank 0 only).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "samples/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0}
SINGLE = ("lidar1m", "room100k", "uniform4k")
L2_NOTE = "GPU arm: L2 flushed between timed steps (256 MiB write)"


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lidar1m", choices=["lidar1m", "room100k", "uniform4k", "batch64", "serving"])
    ap.add_argument("--secondary", default="uniform4k,room100k,batch64,serving",
                    help="comma list of extra workloads measured into the same line (N = 1 only), or 'none'")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: offered clouds per second")
    ap.add_argument("--requests", type=int, default=1500, help="serving: timed requests")
    ap.add_argument("--slots", type=int, default=32, help="serving: micro-batches in flight (one stream each)")
    ap.add_argument("--max-batch", type=int, default=8, help="serving: clouds per micro-batch")
    ap.add_argument("--opts", default="", help="JSON dict of rfps_opts overrides")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="single-cloud workloads: the library's default launch shape instead of the autotuner's")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--floor-sweep", action="store_true",
                    help="print the sampling loop's per-iteration synchronisation floor for every launch shape")
    ap.add_argument("--study", choices=["m-sweep", "ablation", "nvox"],
                    help="latency / memory vs M, prune-skip ablation, or voxel-resolution sensitivity on --workload")
    ap.add_argument("--once", action="store_true",
                    help="run the path once on the workload and exit (the case profiled with ncu)")
    ap.add_argument("--cpu-timing", action="store_true", help=argparse.SUPPRESS)   # the CPU-baseline subprocess
    return ap.parse_args(argv)


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return PEAKS_FALLBACK["hbm_gbs"], "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms; only readings that arrive inside the
    timed region (between mark() and stop()) count.  A timed region shorter than the sampling
    interval may see none: then the last reading before it and the first one after it are taken,
    and the result says so ("window": "adjacent")."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []   # (host time the reading arrived, csv line)
        self.t0 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            deadline = time.time() + 5.0   # the first reading before the timed region starts
            while not self.lines and time.time() < deadline and self.proc.poll() is None:
                time.sleep(0.01)
        except FileNotFoundError:
            self.proc = None

    def mark(self):
        """Start of the timed region."""
        self.t0 = time.time()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        t1 = time.time()
        t0 = self.t0 if self.t0 is not None else 0.0
        adjacent = not any(t0 <= ts <= t1 for ts, _ in self.lines)
        if adjacent:   # wait for the first reading after the timed region
            deadline = time.time() + 0.5
            while not any(ts > t1 for ts, _ in list(self.lines)) and time.time() < deadline:
                time.sleep(0.01)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        if adjacent:
            before = [ln for ts, ln in self.lines if ts < t0][-1:]
            after = [ln for ts, ln in self.lines if ts > t1][:1]
            inside = before + after
        else:
            inside = [ln for ts, ln in self.lines if t0 <= ts <= t1]
        for ln in inside:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "window": "adjacent" if adjacent else "timed"}


# What the autotuner searches (paper_2606_06255_gb300.autotune.candidate_space(); a CPU test keeps the
# two in step).  Stated here so that both arms print the same config without loading the library.
TUNER_SPACE = ("stage 1: 33 launch shapes (cluster 1-16, threads 128/256/512, chunk 64/128/256) at the automatic "
               "resolution; stage 2: the best 2 shapes x nvox_scale [35, 50, 70, 100, 140] "
               "(n_vox = scale/100 * cbrt(N) per cloud)")


def kernel_hash():
    h = hashlib.sha256()
    for f in ("rfps_sample.cu", "rfps_common.cuh"):
        with open(os.path.join(ROOT, "paper_2606_06255_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload, opts):
    """DRAM bytes per launch of the sampling kernel from the committed ncu summary, if it is of the
    current kernel source and the same launch options."""
    p = os.path.join(ROOT, "profiles", f"k_sample_{workload}.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    for cap in d.get("captures", [d]):   # one capture, or several launch shapes of the workload
        if cap.get("kernel_hash") == kernel_hash() and (cap.get("opts") or None) == (opts or None):
            return cap.get("dram_bytes_per_launch")
    return None


def workload_config(name, seed=0):
    """(clouds, config dict) of a workload; both arms print this config."""
    import cloudgen
    if name == "serving":
        return None, {"workload": "serving", "sizes": "N log-uniform [20000, 1200000], M = N/8, half room / half LiDAR",
                      "arrivals": "Poisson", "l2": L2_NOTE}
    clouds, desc = cloudgen.workload(name, seed=seed)
    if name == "batch64":
        return clouds, {"workload": name, "desc": desc, "clouds": len(clouds),
                        "points": int(sum(c.points.shape[0] for c in clouds)), "samples": int(sum(c.m for c in clouds)),
                        "l2": L2_NOTE, "autotune_space": TUNER_SPACE}
    c = clouds[0]
    return clouds, {"workload": name, "desc": desc, "n": int(c.points.shape[0]), "m": int(c.m), "start": int(c.start),
                    "clouds_per_gpu_per_step": 1, "l2": L2_NOTE, "autotune_space": TUNER_SPACE}


def time_oracle(cloud, budget_s=10.0, max_s=30.0, threads=0):
    """The oracle as it stands (plain FPS, every host core by default) on the full workload, repeated ~10 s."""
    import oracle
    reps, t_total = 0, 0.0
    while t_total < budget_s and reps < 1000:
        t0 = time.perf_counter()
        oracle.fps(cloud.points, cloud.m, cloud.start, threads=threads)
        t_total += time.perf_counter() - t0
        reps += 1
        if t_total > max_s:
            break
    return reps, t_total


def placement():
    return {"host": platform.machine(), "cpus": os.cpu_count(),
            "omp_proc_bind": os.environ.get("OMP_PROC_BIND", "unset (threads not pinned)"),
            "omp_num_threads": os.environ.get("OMP_NUM_THREADS", "unset (one per core)")}


def cpu_timing(name, budget_s=10.0):
    """The three CPU timings of the oracle on one single-cloud workload (run in a process of its own
    that has no CUDA context): plain FPS with OpenMP over full runs, plain FPS on one thread over the
    first samples (its per-iteration cost is the same at every step), and the CPU RadiusFPS of
    Sec. 3.2-3.4 on one thread over a full run at the paper's v = 32."""
    import oracle
    clouds, _ = workload_config(name)
    cloud = clouds[0]
    n, m = cloud.points.shape[0], cloud.m
    threads = oracle.openmp_threads() or 1
    reps, secs = time_oracle(cloud, budget_s)
    m1 = min(m, 1024)

    def median_s(fn, k=3):
        ts = []
        for _ in range(k):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        return statistics.median(ts)
    t1 = median_s(lambda: oracle.fps(cloud.points, m1, cloud.start, threads=1))
    t2 = median_s(lambda: oracle.radiusfps(cloud.points, m, cloud.start, n_vox=32))
    plain1 = m1 / t1
    return {
        "value": reps * m / secs, "unit": "samples/s", "cores": threads, "kind": "oracle",
        "sample": f"{reps} full run(s) of the {name} workload (N={n}, M={m}), plain FPS oracle with OpenMP, "
                  f"{secs:.1f} s, in a separate process without a CUDA context",
        "placement": placement(),
        "plain_1thread": {"value": plain1, "unit": "samples/s", "cores": 1,
                          "sample": f"the first {m1} of the {m} samples, median of 3 runs ({t1:.2f} s; plain FPS "
                                    "costs the same per sample at every step)"},
        "radiusfps_1thread": {"value": m / t2, "unit": "samples/s", "cores": 1, "n_vox": 32,
                              "sample": f"full runs, median of 3 ({t2:.2f} s), CPU RadiusFPS oracle (prune + skip)",
                              "speedup_vs_plain_1thread": (m / t2) / plain1},
    }


def cpu_baseline_subprocess(name):
    """cpu_timing() in a fresh interpreter (no torch, no CUDA context); None if it fails."""
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-timing", "--workload", name],
                           capture_output=True, text=True, timeout=600)
        if r.returncode != 0:
            return {"error": (r.stderr or r.stdout)[-300:]}
        return json.loads(r.stdout.strip().splitlines()[-1])
    except (subprocess.TimeoutExpired, ValueError, IndexError) as e:
        return {"error": str(e)}


def run_reference(args, rank):
    """The oracle (plain FPS, every host core) as the reference arm: K timed steps of the same
    workload and config as the GPU arm, on rank 0 only."""
    if rank != 0:
        return 0
    import oracle
    clouds, config = workload_config(args.workload)
    threads = oracle.openmp_threads() or 1
    if clouds is None:   # serving: a bounded sample of the serving stream's clouds, one after another
        import cloudgen
        reqs = cloudgen.serving_requests(4, seed=0)
        clouds = [c for _, c in reqs]
    unit = "samples/s" if args.workload in SINGLE else "clouds/s"
    step_clouds = clouds[:1] if args.workload in SINGLE else clouds
    for _ in range(min(args.warmup, 1)):
        oracle.fps(step_clouds[0].points, step_clouds[0].m, step_clouds[0].start, threads=0)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for c in step_clouds:
            oracle.fps(c.points, c.m, c.start, threads=0)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    per_step = step_clouds[0].m if unit == "samples/s" else len(step_clouds)
    value = per_step / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC if unit == "samples/s" else "clouds/s", "value": value, "unit": unit,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": value, "unit": unit, "cores": threads, "kind": "oracle",
                         "sample": f"full {args.workload} workload per step (plain FPS oracle, OpenMP)",
                         "placement": placement()},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _events(torch, fn, reps, flush):
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def run_study(args, rf, torch, cloud, pts, opts):
    """Secondary studies on one cloud (each row: RadiusFPS vs the plain baselines, same GB300)."""
    n = cloud.points.shape[0]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    base = dict(opts or {})

    def t_fps(m, o, reps=3):
        ws = torch.empty(rf.workspace_size(n, o), dtype=torch.uint8, device="cuda")
        out = torch.empty(m, dtype=torch.int64, device="cuda")
        rf.fps(pts, m, 0, opts=o, workspace=ws, out=out)
        return _events(torch, lambda: rf.fps(pts, m, 0, opts=o, workspace=ws, out=out), reps, flush), ws.numel()

    def t_plain(m, v, reps=2):
        ws = torch.empty(rf.plain_workspace_size(n), dtype=torch.uint8, device="cuda")
        out = torch.empty(m, dtype=torch.int64, device="cuda")
        rf.plain_fps(pts, m, 0, variant=v, workspace=ws, out=out)
        return _events(torch, lambda: rf.plain_fps(pts, m, 0, variant=v, workspace=ws, out=out), reps, flush)

    rows = []
    if args.study == "m-sweep":
        for frac in (1 / 64, 1 / 32, 1 / 16, 1 / 8, 1 / 4):
            m = max(1, int(n * frac))
            ms, wsb = t_fps(m, base or None)
            best_plain = min(t_plain(m, 1), t_plain(m, 2))
            rows.append({"m": m, "ms": ms, "mpts_per_s": n / ms / 1e3, "workspace_mb": wsb / 2**20,
                         "input_mb": n * 12 / 2**20, "plain_best_ms": best_plain, "speedup": best_plain / ms})
    elif args.study == "ablation":
        m = cloud.m
        for prune, skip in ((1, 1), (1, 0), (0, 1), (0, 0)):
            o = dict(base, prune=prune, skip=skip)
            ms, _ = t_fps(m, o)
            cws = torch.empty(rf.workspace_size(n, dict(o, counters=1)), dtype=torch.uint8, device="cuda")
            rf.fps(pts, m, 0, opts=dict(o, counters=1), workspace=cws)
            rows.append({"prune": prune, "skip": skip, "ms": ms, "counters": rf.counters(cws)})
        rows.append({"plain_cluster_ms": t_plain(m, 1), "plain_whole_gpu_ms": t_plain(m, 2)})
    else:
        m = cloud.m
        for nv in (8, 12, 16, 24, 32, 48, 64, 96):
            ms, _ = t_fps(m, dict(base, n_vox=nv))
            rows.append({"n_vox": nv, "ms": ms})
    print(json.dumps({"study": args.study, "workload": args.workload, "n": n, "opts": base or "default",
                      "rows": rows}), flush=True)
    return 0


def measure_batch64(args, rf, torch, world=1, rank=0):
    """64 ragged clouds: one graph-replayed batched launch vs 64 per-cloud launches vs plain batched.

    Under torchrun the clouds are sharded over the ranks (largest work first, no data-path
    collective); each rank samples its share as one batch, and the batch time is the slowest
    rank's (strong scaling: the 64 clouds are the whole job).  Returns the result dict on rank 0
    (None on the other ranks)."""
    from paper_2606_06255_gb300 import shard
    all_clouds, config = workload_config("batch64")
    mine = shard.my_clouds([c.points.shape[0] for c in all_clouds], [c.m for c in all_clouds], world, rank)
    clouds = [all_clouds[b] for b in mine]
    sizes = [c.points.shape[0] for c in clouds]
    ms = [c.m for c in clouds]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    tuned = split_tuned = None
    split = None
    if args.opts:
        opts = single_opts = json.loads(args.opts)
    else:
        # launch shape and automatic-resolution scale picked by the autotuner on this batch (the
        # voxel resolution follows each cloud's size); every candidate gives the same indices
        cat0 = torch.from_numpy(np.ascontiguousarray(np.concatenate([c.points for c in clouds]), np.float32)).cuda()
        single_opts, table = rf.autotune.tune_batch(cat0, sizes, ms, reps=2)
        tuned = [{"ms": round(t, 3), "opts": o} for t, o in table[:8]]
        del cat0
        # then the single launch against size splits (the largest clouds in a concurrent launch)
        (opts, split), stable = rf.autotune.tune_batch_split([c.points for c in clouds], sizes, ms, single_opts)
        split_tuned = [{"ms": round(t, 3), "opts": o, "split": sp} for t, o, sp in stable[:6]]
    bs = rf.batch.BatchSampler(sizes, ms, opts=opts, split=split)
    bs.load([c.points for c in clouds])
    for _ in range(max(args.warmup, 3)):
        bs.run()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    t_batch = _events(torch, bs.run, args.steps, flush)
    launches = bs.kernels_per_run
    if world > 1:
        t = torch.tensor([t_batch], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_batch = float(t.item())
        if rank != 0:
            return None
        return {"metric": "clouds/s", "value": len(all_clouds) / (t_batch / 1e3), "unit": "clouds/s",
                "config": config, "n_gpus": world, "scaling": "strong", "clouds_rank0": len(clouds),
                "ms_per_batch": t_batch, "samples_per_s": sum(c.m for c in all_clouds) / (t_batch / 1e3),
                "opts_rank0": opts, "split_rank0": split, "graph": True,
                "gpu_launches_per_batch_rank0": launches}
    ref = np.concatenate(bs.split())   # the caller's cloud order
    cat = torch.from_numpy(np.ascontiguousarray(np.concatenate([c.points for c in clouds]), np.float32)).cuda()
    meta = rf._lib._batch_meta(sizes, ms, None, cat.device)
    off = meta[3]
    views = [cat[int(off[b]):int(off[b + 1])] for b in range(len(sizes))]
    wss = [torch.empty(rf.workspace_size(sizes[b], single_opts), dtype=torch.uint8, device="cuda")
           for b in range(len(sizes))]
    outs = [torch.empty(ms[b], dtype=torch.int64, device="cuda") for b in range(len(sizes))]

    def per_cloud():
        for b in range(len(sizes)):
            rf.fps(views[b], ms[b], 0, opts=single_opts, workspace=wss[b], out=outs[b])
    per_cloud()
    t_sep = _events(torch, per_cloud, 2, flush)
    same = bool(np.array_equal(np.concatenate([o.cpu().numpy() for o in outs]), ref))
    plain = {}
    pws = torch.empty(rf.plain_workspace_size(cat.shape[0], len(sizes)), dtype=torch.uint8, device="cuda")
    for v in (1, 0):
        res = {}
        t = _events(torch, lambda: res.setdefault("o", rf.plain_fps_batched(cat, sizes, ms, variant=v, workspace=pws,
                                                                           meta=meta)[0]), 1, flush)
        plain[f"variant{v}"] = {"ms": t, "clouds_per_s": len(sizes) / (t / 1e3)}
    return {"metric": "clouds/s", "value": len(sizes) / (t_batch / 1e3), "unit": "clouds/s", "config": config,
            "ms_per_batch": t_batch, "samples_per_s": sum(ms) / (t_batch / 1e3), "opts": opts, "split": split,
            "autotune": tuned, "split_autotune": split_tuned, "graph": True, "gpu_launches_per_batch": launches,
            "per_cloud_launches": {"ms": t_sep, "clouds_per_s": len(sizes) / (t_sep / 1e3), "same_indices": same},
            "batched_vs_per_cloud": t_sep / t_batch, "plain_batched": plain,
            "batched_vs_plain_batched": min(p["ms"] for p in plain.values()) / t_batch}


# size-aware route of the serving run: clouds of TAIL_N points or more (the latency tail) run
# alone on an 8-CTA cluster instead of one CTA each
TAIL_N = 600_000
TAIL_OPTS = {"cluster": 8, "threads": 256}


def measure_serving(args, rf, world=1, rank=0, routed=False):
    """Poisson request stream through the continuous-batching server.  Under torchrun the stream
    is sharded round-robin over the ranks, each serving its share on its own GPU; rank 0 merges
    the outcomes (latency percentiles and throughput over the whole stream).  routed=True adds the
    size-aware route of the largest clouds."""
    from paper_2606_06255_gb300 import serve
    # throughput setting: one CTA of 512 threads per cloud (the most SM-efficient shape), many streams
    opts = json.loads(args.opts) if args.opts else {"cluster": 1, "threads": 512}
    reqs = serve.poisson_workload(args.requests + 16, args.rate, pinned=True)
    ex = serve.GpuExecutor(args.slots, opts=opts, tail_opts=TAIL_OPTS if routed else None,
                           tail_n=TAIL_N if routed else None)
    srv = serve.Server(ex, mem_budget=48 << 30, max_inflight=args.slots, max_batch=args.max_batch)
    srv.run([r for r in reqs[:16] if r.rid % world == rank])
    t0 = reqs[16].arrival
    timed = [serve.Request(r.rid, r.arrival - t0, r.points, r.m, r.start) for r in reqs[16:] if r.rid % world == rank]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    rep = srv.run(timed)
    if world > 1:
        for c in rep.completed:   # the indices stay on their rank; only the outcome travels
            c.indices = None
        parts = [None] * world
        dist.all_gather_object(parts, rep)
        if rank != 0:
            return None
        rep = serve.merge_reports(parts)
    out = rep.summary()
    out["n_gpus"] = world
    out.update({"metric": "p99 latency / clouds/s", "workload": "serving", "offered_rate": args.rate,
                "requests": args.requests, "opts": opts, "slots": args.slots, "max_batch": args.max_batch,
                "sizes": "N log-uniform [20000, 1200000], M = N/8, half room / half LiDAR"})
    if routed:
        out["route"] = {"tail_n": TAIL_N, "tail_opts": TAIL_OPTS}
    return out


def _timed_steps(torch, fn, steps, flush, stream):
    """K steps of fn, each between CUDA events on `stream`, L2 flushed before each (outside the events)."""
    evs = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def measure_single(args, rf, torch, name, world=1, rank=0, local=0, full=True):
    """One single-cloud workload: autotuned launch shape, K timed steps (index build + sampling), the
    sampling kernel alone against its exchange floor, and the plain GPU FPS baselines on the same
    cloud.  full=True (the headline) adds the clock record, work counters, roofline, on-chip probes
    and the end-to-end run through the C ABI with host buffers."""
    dist = None
    if world > 1:
        import torch.distributed as dist
    dev = torch.device("cuda", local)
    clouds, config = workload_config(name, seed=rank)
    cloud = clouds[0]
    n, m, start = cloud.points.shape[0], cloud.m, cloud.start
    opts = json.loads(args.opts) if (args.opts and full) else None
    pts = torch.from_numpy(cloud.points).to(dev)
    tuned = None
    if opts is None and not args.no_tune:
        # launch shape, then voxel resolution, from the autotuner, timed on this cloud before (outside)
        # the timed region; every candidate returns the same indices
        opts, table = rf.autotune.tune_single(pts, m, start, reps=3)
        tuned = [{"ms": round(t, 3), "opts": o} for t, o in table[:10]]
    ws = torch.empty(rf.workspace_size(n, opts), dtype=torch.uint8, device=dev)
    out = torch.empty(m, dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        rf.fps(pts, m, start, opts=opts, workspace=ws, out=out)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if rf.status(ws) != 0:
        raise RuntimeError("device status after warm-up: %d" % rf.status(ws))

    clocks = ClockSampler(local) if full else None
    if clocks:
        clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.mark()
    launches0 = rf.launch_count()
    step_ms = _timed_steps(torch, step, args.steps if full else min(args.steps, 10), flush, stream)
    launches = rf.launch_count() - launches0
    if dist:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / len(step_ms)
    value = world * m / (ms_per_step / 1e3)

    # ---- the sampling kernel alone (index path: tiny re-arm kernel + k_sample) against its exchange floor
    ix = rf.Index(pts, opts=opts)
    n_vox = ix.export()["n_vox"]
    for _ in range(2):
        ix.sample(m, start, out=out)
    k_ms = statistics.mean(_timed_steps(torch, lambda: ix.sample(m, start, out=out), min(args.steps, 5), flush,
                                        stream))
    ix.free()
    rs = rf.resolved_opts(n, opts)
    floor_ms = min(rf.sync_floor(rs["cluster"], rs["threads"], max(2, m)) for _ in range(3))
    ns_iter = k_ms * 1e6 / max(1, m - 1)
    floor_ns = floor_ms * 1e6 / max(1, m - 1)

    # ---- plain GPU FPS on the same cloud: cluster-resident (variant 1), whole GPU (variant 2), one CTA (0)
    plain = None
    if not args.no_plain:
        plain = {}
        pws = torch.empty(rf.plain_workspace_size(n), dtype=torch.uint8, device=dev)
        for variant, label in ((1, "cluster"), (2, "whole_gpu"), (0, "one_cta_per_cloud")):
            rf.plain_fps(pts, m, start, variant=variant, workspace=pws, out=out)
            torch.cuda.synchronize()
            reps = 1 if (variant == 0 and n > 50000) else max(2, min(args.steps, 3))
            pm = statistics.mean(_timed_steps(
                torch, lambda: rf.plain_fps(pts, m, start, variant=variant, workspace=pws, out=out), reps, flush, stream))
            plain[label] = {"variant": variant, "ms_per_cloud": pm, "samples_per_s": m / (pm / 1e3),
                            "radiusfps_speedup": pm / ms_per_step,
                            # 16 B (coordinates + d2) per point per iteration, index build included
                            "achieved_gbs": 16 * n * (m - 1) / (pm / 1e3) / 1e9}
    res = {"config": config, "ms_per_cloud": ms_per_step, "samples_per_s": value, "opts": opts or "default",
           "autotune": tuned, "n_vox": n_vox, "launch_shape": {"cluster": rs["cluster"], "threads": rs["threads"],
                                                               "chunk": rs["chunk"]},
           "kernel_ms": k_ms, "ns_per_iteration": ns_iter, "sync_floor_ns_per_iteration": floor_ns,
           "plain_gpu_fps": plain}
    if plain:
        best = min(plain.values(), key=lambda p: p["ms_per_cloud"])
        res["best_plain"] = {"variant": best["variant"], "ms_per_cloud": best["ms_per_cloud"],
                             "radiusfps_speedup": best["radiusfps_speedup"]}
    # ---- work counters of one sampling launch (untimed counting run): exchange rounds, and the
    # algorithmic bytes below
    cws = torch.empty(rf.workspace_size(n, dict(opts or {}, counters=1)), dtype=torch.uint8, device=dev)
    rf.fps(pts, m, start, opts=dict(opts or {}, counters=1), workspace=cws, out=out)
    c = rf.counters(cws)
    spr = (m - 1) / max(1, c["rounds"])   # samples per exchange round
    res.update({"rounds": c["rounds"], "samples_per_round": spr, "ns_per_round": spr * ns_iter,
                "latency_frac": floor_ns / (spr * ns_iter)})
    if not full:
        return res

    resynced = c["voxel_tests"] - c["voxels_pruned"]
    alg_bytes = 32 * c["voxel_tests"] + 16 * c["points_visited"] + 4 * c["points_updated"] + 8 * resynced
    peak, peak_kind = load_peaks()
    achieved = alg_bytes / (k_ms / 1e3) / 1e9
    # ---- on-chip roofline: after the first touch the loop's bytes come from shared memory and L2,
    # and one cloud occupies one cluster of SMs
    smem_bw = rf.bandwidth_probe("smem")
    l2_bw = rf.bandwidth_probe("l2")
    sms_used = rs["cluster"]
    onchip_peak = smem_bw["gbs_per_sm"] * sms_used
    min_floor_ns = min(rf.sync_floor(1, 128, max(2, m)) for _ in range(3)) * 1e6 / max(1, m - 1)

    # ---- end to end through the C ABI with host buffers (copies inside the timed region)
    host_pts = torch.empty((n, 3), dtype=torch.float32, pin_memory=True)
    host_pts.copy_(torch.from_numpy(cloud.points))
    hws = torch.empty(rf.host_workspace_size(n, opts), dtype=torch.uint8, device=dev)
    hp = host_pts.numpy()
    rf.fps_host(hp, m, start, opts=opts, workspace=hws)
    e2e_s = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rf.fps_host(hp, m, start, opts=opts, workspace=hws)
        e2e_s.append(time.perf_counter() - t0)
    e2e_mean = statistics.mean(e2e_s)
    if dist:   # the slowest rank, as for the device-timed value
        t = torch.tensor([e2e_mean], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_mean = float(t.item())

    line = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": len(step_ms),
        "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config,
        "ms_per_cloud": ms_per_step,
        "launch": {"opts": opts or "default", "n_vox": n_vox, "shape": res["launch_shape"], "autotune": tuned},
        "plain_gpu_fps": plain,
        "best_plain": res.get("best_plain"),
        # The sampling loop is bound by its cluster exchange rounds, not by bandwidth: its headline
        # efficiency is the exchange floor of its launch shape over the time per round.  A round
        # selects one sample, or two when the runner-up shortcut applies (`samples_per_round`, from
        # the counting run), so the bound per sample is the floor over the samples per round.
        "roofline": {"bound": "latency", "achieved": 1e9 / ns_iter, "peak": 1e9 * spr / floor_ns,
                     "unit": "iterations/s", "frac": floor_ns / (spr * ns_iter), "traffic": ncu_traffic(name, opts),
                     "kernel": "k_sample", "kernel_ms": k_ms,
                     "ns_per_iteration": ns_iter, "sync_floor_ns_per_iteration": floor_ns,
                     "rounds": c["rounds"], "samples_per_round": spr, "ns_per_round": spr * ns_iter,
                     "peak_kind": "exchange floor per round of the same launch shape (rfps_sync_floor, measured in "
                                  "this run) over the samples per round",
                     "min_floor_ns_per_iteration": min_floor_ns, "launch_shape": res["launch_shape"],
                     "hbm": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                             "peak_kind": peak_kind, "alg_bytes_per_launch": alg_bytes,
                             "traffic": ncu_traffic(name, opts)},
                     "onchip": {"bound": "smem", "sms_used": sms_used, "achieved": achieved, "peak": onchip_peak,
                                "unit": "GB/s", "frac": achieved / onchip_peak,
                                "smem_gbs_per_sm": smem_bw["gbs_per_sm"], "smem_gbs": smem_bw["gbs"],
                                "l2_gbs": l2_bw["gbs"], "l2_probe_bytes": l2_bw["buffer_bytes"],
                                "peak_kind": "measured by rfps_bandwidth_probe in this run"}},
        "counters": c,
        "cpu_baseline": None,
        "e2e": {"value": world * m / e2e_mean, "unit": "samples/s", "h2d_bytes_per_step": n * 12,
                "d2h_bytes_per_step": m * 8},
        "gpu_launches": launches,
        "clocks": clk,
    }
    return line if rank == 0 else None


def main(argv=None):
    args = parse(argv)
    world, rank, local = dist_setup(args)
    if args.cpu_timing:
        print(json.dumps(cpu_timing(args.workload)), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args, rank)

    import torch
    import torch.distributed as dist

    import paper_2606_06255_gb300 as rf

    torch.cuda.set_device(local)
    if args.floor_sweep:
        for cluster in (1, 2, 4, 8, 16):
            for threads in (128, 256, 512):
                ms = min(rf.sync_floor(cluster, threads, 25000) for _ in range(3))
                print(json.dumps({"cluster": cluster, "threads": threads, "ns_per_iteration": ms * 1e6 / 24999}),
                      flush=True)
        return 0
    if args.study or args.once:
        if args.workload not in SINGLE:
            raise SystemExit("--study / --once take a single-cloud workload")
        (cloud,), _ = workload_config(args.workload)
        pts = torch.from_numpy(cloud.points).cuda()
        opts = json.loads(args.opts) if args.opts else None
        if args.study:
            return run_study(args, rf, torch, cloud, pts, opts)
        ws = torch.empty(rf.workspace_size(pts.shape[0], opts), dtype=torch.uint8, device="cuda")
        out = rf.fps(pts, cloud.m, cloud.start, opts=opts, workspace=ws)
        torch.cuda.synchronize()
        if rf.status(ws) != 0:
            raise RuntimeError("device status %d" % rf.status(ws))
        print(json.dumps({"once": args.workload, "n": pts.shape[0], "m": cloud.m, "first": out[:4].tolist()}),
              flush=True)
        return 0
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload == "batch64":
        line = measure_batch64(args, rf, torch, world, rank)
    elif args.workload == "serving":
        line = measure_serving(args, rf, world, rank)
    else:
        line = measure_single(args, rf, torch, args.workload, world, rank, local, full=True)
    if line is not None and world == 1 and args.secondary != "none":
        # the other configurations, measured into the same line (each with its own timing)
        for name in [s for s in args.secondary.split(",") if s and s != args.workload]:
            if name in SINGLE:
                line[name] = measure_single(args, rf, torch, name, full=False)
            elif name == "batch64":
                line[name] = measure_batch64(args, rf, torch)
            elif name == "serving":
                line[name] = measure_serving(args, rf)
                # the same stream with the largest clouds routed to a 4-CTA cluster each
                line[name]["routed"] = measure_serving(args, rf, routed=True)
    if line is not None and args.workload in SINGLE and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_subprocess(args.workload)   # after the GPU work, in a clean process
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
