"""Benchmark of the RadiusFPS hot path on GB300: one JSON line on rank 0.

A step is one full pass of the path over one cloud: device-side voxel index
build (bounding box, binning, sort, records) plus the persistent sampling
kernel (initial update, then M - 1 select / prune / skip / update / resync
iterations).  Default workload: the room-like cloud, N = 100,000 points,
M = 25,000 samples, start 0 (synthetic stand-in for the paper's indoor
scans).  Other workloads: --workload uniform4k | lidar1m.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events
on the launching stream; between steps a 256 MiB buffer is written to flush
the 129 MB L2 (outside the events).  Barrier + synchronize on both sides of
the timed loop, max over ranks.  Multi-GPU: one process per GPU, each samples
its own cloud (clouds are independent units; no data-path collective).

--impl reference times the CPU oracle (plain FPS, all host cores) on the
same workload instead (rank 0 only).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="room100k",
                    choices=["room100k", "uniform4k", "lidar1m", "batch64", "serving"])
    ap.add_argument("--rate", type=float, default=200.0, help="serving: offered clouds per second")
    ap.add_argument("--requests", type=int, default=600, help="serving: timed requests")
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
    return ap.parse_args()


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


# launch shapes the single-cloud benchmark lets the autotuner choose between
TUNE_CANDIDATES = [{"cluster": 16, "threads": 256}, {"cluster": 16, "threads": 128}, {"cluster": 8, "threads": 256},
                   {"cluster": 16, "threads": 256, "chunk": 256}]


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
    if d.get("kernel_hash") != kernel_hash() or (d.get("opts") or None) != (opts or None):
        return None
    return d.get("dram_bytes_per_launch")


def cpu_threads():
    import oracle
    return oracle.openmp_threads() or 1


def time_oracle(cloud, budget_s=10.0, max_s=30.0):
    """The oracle as it stands (plain FPS, every host core) on the full workload, repeated ~10 s."""
    import oracle
    reps, t_total = 0, 0.0
    while t_total < budget_s and reps < 1000:
        t0 = time.perf_counter()
        oracle.fps(cloud.points, cloud.m, cloud.start, threads=0)
        t_total += time.perf_counter() - t0
        reps += 1
        if t_total > max_s:
            break
    return reps, t_total


def run_reference(args, rank):
    if rank != 0:
        return 0
    import cloudgen
    (cloud,), desc = cloudgen.workload(args.workload, seed=0)
    threads = cpu_threads()
    # warm-up, then K timed steps; each step one full oracle run of the workload
    for _ in range(min(args.warmup, 1)):
        time_oracle(cloud, budget_s=0.0)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        import oracle
        oracle.fps(cloud.points, cloud.m, cloud.start, threads=0)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    value = cloud.m / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "desc": desc, "n": int(cloud.points.shape[0]), "m": cloud.m},
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": threads, "kind": "oracle",
                         "sample": f"full {args.workload} workload per step (plain FPS oracle, OpenMP)"},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
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


def run_batch64(args, rf, torch, world=1, rank=0):
    """64 ragged clouds: one graph-replayed batched launch vs 64 per-cloud launches vs plain batched.

    Under torchrun the clouds are sharded over the ranks (largest work first, no data-path
    collective); each rank samples its share as one batch, and the batch time is the slowest
    rank's (strong scaling: the 64 clouds are the whole job)."""
    import cloudgen
    from paper_2606_06255_gb300 import shard
    all_clouds, desc = cloudgen.workload("batch64")
    mine = shard.my_clouds([c.points.shape[0] for c in all_clouds], [c.m for c in all_clouds], world, rank)
    clouds = [all_clouds[b] for b in mine]
    sizes = [c.points.shape[0] for c in clouds]
    ms = [c.m for c in clouds]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    tuned = None
    if args.opts:
        opts = json.loads(args.opts)
    else:
        # launch shape picked by the autotuner on this batch (cluster size, CTA threads, record
        # chunk; the voxel resolution follows each cloud's size); every candidate gives the same indices
        cat0 = torch.from_numpy(np.ascontiguousarray(np.concatenate([c.points for c in clouds]), np.float32)).cuda()
        opts, table = rf.autotune.tune_batch(cat0, sizes, ms, reps=2)
        tuned = [{"ms": round(t, 3), "opts": o} for t, o in table]
        del cat0
    bs = rf.batch.BatchSampler(sizes, ms, opts=opts)
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
        if rank == 0:
            print(json.dumps({
                "metric": "clouds/s", "value": len(all_clouds) / (t_batch / 1e3), "unit": "clouds/s",
                "workload": "batch64", "desc": desc, "n_gpus": world, "scaling": "strong",
                "clouds": len(all_clouds), "clouds_rank0": len(clouds), "ms_per_batch": t_batch,
                "samples_per_s": sum(c.m for c in all_clouds) / (t_batch / 1e3), "opts_rank0": opts,
                "graph": True, "gpu_launches_per_batch_rank0": launches}), flush=True)
        return 0
    ref = bs.out.cpu().numpy()
    cat, off = bs.points, bs.offsets
    views = [cat[int(off[b]):int(off[b + 1])] for b in range(len(sizes))]
    wss = [torch.empty(rf.workspace_size(sizes[b], opts), dtype=torch.uint8, device="cuda") for b in range(len(sizes))]
    outs = [torch.empty(ms[b], dtype=torch.int64, device="cuda") for b in range(len(sizes))]

    def per_cloud():
        for b in range(len(sizes)):
            rf.fps(views[b], ms[b], 0, opts=opts, workspace=wss[b], out=outs[b])
    per_cloud()
    t_sep = _events(torch, per_cloud, 2, flush)
    same = bool(np.array_equal(np.concatenate([o.cpu().numpy() for o in outs]), ref))
    plain = {}
    pws = torch.empty(rf.plain_workspace_size(cat.shape[0], len(sizes)), dtype=torch.uint8, device="cuda")
    for v in (1, 0):
        res = {}
        t = _events(torch, lambda: res.setdefault("o", rf.plain_fps_batched(cat, sizes, ms, variant=v, workspace=pws,
                                                                           meta=bs.meta)[0]), 1, flush)
        plain[f"variant{v}"] = {"ms": t, "clouds_per_s": len(sizes) / (t / 1e3)}
    print(json.dumps({
        "metric": "clouds/s", "value": len(sizes) / (t_batch / 1e3), "unit": "clouds/s", "workload": "batch64",
        "desc": desc, "clouds": len(sizes), "points": int(sum(sizes)), "samples": int(sum(ms)),
        "ms_per_batch": t_batch, "samples_per_s": sum(ms) / (t_batch / 1e3), "opts": opts, "autotune": tuned,
        "graph": True,
        "gpu_launches_per_batch": launches,
        "per_cloud_launches": {"ms": t_sep, "clouds_per_s": len(sizes) / (t_sep / 1e3), "same_indices": same},
        "batched_vs_per_cloud": t_sep / t_batch, "plain_batched": plain}), flush=True)
    return 0


def run_serving(args, rf, world=1, rank=0):
    """Poisson request stream through the continuous-batching server.  Under torchrun the stream
    is sharded round-robin over the ranks, each serving its share on its own GPU; rank 0 merges
    the outcomes (latency percentiles and throughput over the whole stream)."""
    from paper_2606_06255_gb300 import serve
    # throughput setting: one CTA of 512 threads per cloud (the most SM-efficient shape), many streams
    opts = json.loads(args.opts) if args.opts else {"cluster": 1, "threads": 512}
    reqs = serve.poisson_workload(args.requests + 16, args.rate, pinned=True)
    ex = serve.GpuExecutor(args.slots, opts=opts)
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
            return 0
        rep = serve.merge_reports(parts)
    out = rep.summary()
    out["n_gpus"] = world
    out.update({"metric": "p99 latency / clouds/s", "workload": "serving", "offered_rate": args.rate,
                "requests": args.requests, "opts": opts, "slots": args.slots, "max_batch": args.max_batch,
                "sizes": "N log-uniform [20000, 1200000], M = N/8, half room / half LiDAR"})
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, rank)

    import torch
    import torch.distributed as dist

    import cloudgen
    import paper_2606_06255_gb300 as rf

    torch.cuda.set_device(local)
    if args.floor_sweep:
        for cluster in (1, 2, 4, 8, 16):
            for threads in (128, 256, 512):
                ms = min(rf.sync_floor(cluster, threads, 25000) for _ in range(3))
                print(json.dumps({"cluster": cluster, "threads": threads, "ns_per_iteration": ms * 1e6 / 24999}),
                      flush=True)
        return 0
    if world > 1 and not args.floor_sweep:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload == "batch64":
        rc = run_batch64(args, rf, torch, world, rank)
    elif args.workload == "serving":
        rc = run_serving(args, rf, world, rank)
    else:
        rc = None
    if rc is not None:
        if world > 1:
            dist.destroy_process_group()
        return rc
    dev = torch.device("cuda", local)
    (cloud,), desc = cloudgen.workload(args.workload, seed=rank)
    n, m, start = cloud.points.shape[0], cloud.m, cloud.start
    opts = json.loads(args.opts) if args.opts else None
    pts = torch.from_numpy(cloud.points).to(dev)
    tuned = None
    if opts is None and not (args.no_tune or args.once or args.study):
        # launch shape from the autotuner, timed on this cloud before (outside) the timed region;
        # every candidate returns the same indices
        opts, table = rf.autotune.tune_single(pts, m, start, candidates=TUNE_CANDIDATES, reps=3)
        tuned = [{"ms": round(t, 3), "opts": o} for t, o in table]
    ws = torch.empty(rf.workspace_size(n, opts), dtype=torch.uint8, device=dev)
    out = torch.empty(m, dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        rf.fps(pts, m, start, opts=opts, workspace=ws, out=out)

    if args.study:
        return run_study(args, rf, torch, cloud, pts, opts)

    if args.once:
        step()
        torch.cuda.synchronize()
        if rf.status(ws) != 0:
            raise RuntimeError("device status %d" % rf.status(ws))
        print(json.dumps({"once": args.workload, "n": n, "m": m, "first": out[:4].tolist()}), flush=True)
        return 0

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if rf.status(ws) != 0:
        raise RuntimeError("device status after warm-up: %d" % rf.status(ws))

    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark()
    launches0 = rf.launch_count()
    evs = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    launches = rf.launch_count() - launches0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * args.steps * m / (total_ms / 1e3)

    # ---- the sampling kernel alone (index path: tiny re-arm kernel + k_sample), for the roofline
    ix = rf.Index(pts, opts=opts)
    for _ in range(2):
        ix.sample(m, start, out=out)
    sample_ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ix.sample(m, start, out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        sample_ms.append(e0.elapsed_time(e1))
    ix.free()
    k_ms = statistics.mean(sample_ms)

    # ---- algorithmic bytes of one sampling launch, from the work counters (untimed run)
    cws = torch.empty(rf.workspace_size(n, dict(opts or {}, counters=1)), dtype=torch.uint8, device=dev)
    rf.fps(pts, m, start, opts=dict(opts or {}, counters=1), workspace=cws, out=out)
    c = rf.counters(cws)
    resynced = c["voxel_tests"] - c["voxels_pruned"]
    alg_bytes = 32 * c["voxel_tests"] + 16 * c["points_visited"] + 4 * c["points_updated"] + 8 * resynced
    peak, peak_kind = load_peaks()
    achieved = alg_bytes / (k_ms / 1e3) / 1e9

    # ---- per-iteration synchronisation floor of the launch shape the step used
    rs = rf.resolved_opts(n, opts)
    # ---- on-chip roofline: after the first touch the loop's bytes come from shared memory and L2,
    # and one cloud occupies one cluster of SMs
    smem_bw = rf.bandwidth_probe("smem")
    l2_bw = rf.bandwidth_probe("l2")
    sms_used = rs["cluster"]
    onchip_peak = smem_bw["gbs_per_sm"] * sms_used
    floor_ms = min(rf.sync_floor(rs["cluster"], rs["threads"], max(2, m)) for _ in range(3))
    floor_ns = floor_ms * 1e6 / max(1, m - 1)

    # ---- plain GPU FPS on the same cloud: cluster-resident (variant 1) and whole-GPU (variant 2)
    plain = None
    if not args.no_plain:
        plain = {}
        pws = torch.empty(rf.plain_workspace_size(n), dtype=torch.uint8, device=dev)
        for variant, label in ((1, "cluster"), (2, "whole_gpu"), (0, "one_cta_per_cloud")):
            rf.plain_fps(pts, m, start, variant=variant, workspace=pws, out=out)
            torch.cuda.synchronize()
            p_ms = []
            for _ in range(1 if variant == 0 else max(2, min(args.steps, 3))):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rf.plain_fps(pts, m, start, variant=variant, workspace=pws, out=out)
                e1.record(stream)
                torch.cuda.synchronize()
                p_ms.append(e0.elapsed_time(e1))
            pm = statistics.mean(p_ms)
            plain[label] = {"variant": variant, "ms_per_cloud": pm, "samples_per_s": m / (pm / 1e3),
                            "radiusfps_speedup": pm / ms_per_step,
                            # 16 B (coordinates + d2) per point per iteration, index build included
                            "achieved_gbs": 16 * n * (m - 1) / (pm / 1e3) / 1e9}

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
    if world > 1:   # the slowest rank, as for the device-timed value
        t = torch.tensor([e2e_mean], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_mean = float(t.item())
    e2e_value = world * m / e2e_mean

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        reps, secs = time_oracle(cloud)
        cpu = {"value": reps * m / secs, "unit": "samples/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"{reps} full run(s) of the {args.workload} workload (N={n}, M={m}), "
                         f"plain FPS oracle with OpenMP, {secs:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "desc": desc, "n": n, "m": m, "start": start,
                       "clouds_per_gpu_per_step": 1, "l2": "flushed between steps (256 MiB write)",
                       "opts": opts or "default", "autotune": tuned},
            "ms_per_cloud": ms_per_step,
            "plain_gpu_fps": plain,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": ncu_traffic(args.workload, opts),
                         "kernel": "k_sample", "kernel_ms": k_ms, "alg_bytes_per_launch": alg_bytes,
                         "peak_kind": peak_kind,
                         "ns_per_iteration": k_ms * 1e6 / max(1, m - 1),
                         "sync_floor_ns_per_iteration": floor_ns,
                         "launch_shape": {"cluster": rs["cluster"], "threads": rs["threads"]},
                         "onchip": {"bound": "smem", "sms_used": sms_used, "peak": onchip_peak, "unit": "GB/s",
                                    "frac": achieved / onchip_peak,
                                    "smem_gbs_per_sm": smem_bw["gbs_per_sm"], "smem_gbs": smem_bw["gbs"],
                                    "l2_gbs": l2_bw["gbs"], "l2_probe_bytes": l2_bw["buffer_bytes"],
                                    "peak_kind": "measured by rfps_bandwidth_probe in this run"}},
            "counters": c,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "samples/s", "h2d_bytes_per_step": n * 12,
                    "d2h_bytes_per_step": m * 8},
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
