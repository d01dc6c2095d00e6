"""Host-side logic without a GPU: serving scheduler (simulated executor) and
multi-rank sharding (world size 2 over gloo)."""

import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import cloudgen
import oracle

from paper_2606_06255_gb300 import serve, shard


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-5)


class SimExecutor:
    """Runs the oracle on launch and completes after a simulated duration."""

    def __init__(self, clock, per_sample_s=1e-6, bytes_per_point=100):
        self.clock = clock
        self.per_sample = per_sample_s
        self.bpp = bytes_per_point
        self.launched = []

    def mem_needed(self, batch):
        return sum(r.points.shape[0] for r in batch) * self.bpp

    def launch(self, batch, slot):
        self.launched.append([r.rid for r in batch])
        res = []
        for r in batch:
            if r.more_of is not None:     # continue the kept sequence: the slice of a longer run
                pts, start, taken = self.kept[r.more_of]
                res.append(oracle.fps(pts, taken + r.m, start)[taken:])
            else:
                res.append(oracle.fps(r.points, r.m, r.start))
        dur = max(r.m for r in batch) * self.per_sample
        return {"t_done": self.clock() + dur, "res": res, "batch": batch}

    def done(self, h):
        return self.clock() >= h["t_done"]

    def results(self, h):
        for r in h["batch"]:
            if r.more_of is not None:
                pts, start, taken = self.kept.pop(r.more_of)
                self.kept[r.rid] = (pts, start, taken + r.m)
            elif r.keep:
                self.kept[r.rid] = (r.points, r.start, r.m)
        return h["res"]

    # kept indices (follow-up requests)
    kept_size = 10_000

    @property
    def kept(self):
        if not hasattr(self, "_kept"):
            self._kept = {}
            self.released = []
        return self._kept

    def kept_bytes(self, rid):
        return self.kept_size if rid in self.kept else 0

    def release(self, rid):
        self.kept.pop(rid, None)
        self.released.append(rid)


def _requests(n, rate, seed=0):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    reqs = []
    for i in range(n):
        pts = cloudgen.uniform_cloud(int(rng.integers(200, 2000)), seed=100 + i)
        reqs.append(serve.Request(i, float(t[i]), pts, max(1, pts.shape[0] // 8), int(rng.integers(0, 10))))
    return reqs


def test_scheduler_completes_everything_with_exact_results():
    clk = FakeClock()
    ex = SimExecutor(clk)
    reqs = _requests(40, rate=2000.0)
    rep = serve.Server(ex, mem_budget=400_000, max_inflight=3, max_batch=4).run(reqs, clock=clk, sleep=clk.sleep)
    assert len(rep.completed) == 40 and not rep.rejected
    by_id = {c.rid: c for c in rep.completed}
    for r in reqs:
        c = by_id[r.rid]
        np.testing.assert_array_equal(c.indices, oracle.fps(r.points, r.m, r.start))
        assert c.admitted >= r.arrival and c.finished >= c.admitted
    s = rep.summary()
    assert s["p99_latency_ms"] >= s["p50_latency_ms"] > 0
    assert rep.max_inflight_batches <= 3
    assert rep.peak_mem <= 400_000
    assert max(len(b) for b in ex.launched) <= 4
    # continuous batching: later arrivals were admitted while earlier batches ran
    assert rep.max_inflight_batches >= 2


def test_scheduler_admits_by_memory_and_rejects_oversize():
    clk = FakeClock()
    ex = SimExecutor(clk, bytes_per_point=1000)
    reqs = _requests(10, rate=5000.0, seed=3)
    big = serve.Request(99, 0.0005, cloudgen.uniform_cloud(5000, seed=7), 10)
    rep = serve.Server(ex, mem_budget=2_500_000, max_inflight=4, max_batch=8).run(reqs + [big], clock=clk,
                                                                                 sleep=clk.sleep)
    assert rep.rejected == [99]
    assert len(rep.completed) == 10
    assert rep.peak_mem <= 2_500_000


class FlakyExecutor(SimExecutor):
    """Launches fail (an allocation error) or report a device error on chosen requests."""

    def __init__(self, clock, launch_fail, result_fail, **kw):
        super().__init__(clock, **kw)
        self.launch_fail = dict(launch_fail)     # rid -> failing launches left
        self.result_fail = dict(result_fail)

    def launch(self, batch, slot):
        for r in batch:
            if self.launch_fail.get(r.rid, 0) > 0:
                self.launch_fail[r.rid] -= 1
                raise MemoryError("simulated allocation failure")
        h = super().launch(batch, slot)
        h["bad"] = any(self.result_fail.get(r.rid, 0) > 0 for r in batch)
        for r in batch:
            if self.result_fail.get(r.rid, 0) > 0:
                self.result_fail[r.rid] -= 1
        return h

    def results(self, h):
        if h["bad"]:
            raise RuntimeError("device status 5")
        return super().results(h)


def test_failed_batches_are_retried_then_reported():
    clk = FakeClock()
    reqs = _requests(30, rate=3000.0, seed=11)
    # rid 3: one failed launch (retried, then served); rid 7: launches always fail; rid 12: one
    # device error (retried); rid 20: device errors every time
    ex = FlakyExecutor(clk, launch_fail={3: 1, 7: 99}, result_fail={12: 1, 20: 99})
    rep = serve.Server(ex, mem_budget=10**9, max_inflight=3, max_batch=4, max_retries=2).run(
        reqs, clock=clk, sleep=clk.sleep)
    failed = {rid for rid, _ in rep.failed}
    assert failed == {7, 20}
    assert all("launch" in why for rid, why in rep.failed if rid == 7)
    assert all("results" in why for rid, why in rep.failed if rid == 20)
    done = {c.rid: c for c in rep.completed}
    assert set(done) == {r.rid for r in reqs} - failed   # batch-mates of failing requests are served too
    for r in reqs:
        if r.rid in done:
            np.testing.assert_array_equal(done[r.rid].indices, oracle.fps(r.points, r.m, r.start))
    assert rep.summary()["requests_failed"] == 2


def test_deadlines_and_cancellation_while_queued():
    clk = FakeClock()
    ex = SimExecutor(clk, per_sample_s=2e-4)         # slow: the queue builds up behind one slot
    reqs = _requests(12, rate=10000.0, seed=13)
    reqs[5].deadline = 1e-3                          # cannot be admitted that soon
    reqs[8].cancel_at = reqs[8].arrival + 1e-4       # withdrawn while still queued
    reqs[10].deadline = 1e3                          # generous: served
    rep = serve.Server(ex, mem_budget=10**9, max_inflight=1, max_batch=1).run(reqs, clock=clk, sleep=clk.sleep)
    assert rep.expired == [5] and rep.cancelled == [8]
    done = {c.rid for c in rep.completed}
    assert done == {r.rid for r in reqs} - {5, 8}
    s = rep.summary()
    assert s["requests_expired"] == 1 and s["requests_cancelled"] == 1


def test_assignment_balances_and_covers():
    sizes = [8000, 200000, 50000, 12000, 90000, 30000, 150000, 9000]
    ms = [n // 4 for n in sizes]
    shards = shard.assign(sizes, ms, 3)
    flat = sorted(b for s in shards for b in s)
    assert flat == list(range(len(sizes)))
    assert shard.assign(sizes, ms, 3) == shards          # deterministic
    loads = [sum(sizes[b] * ms[b] for b in s) for s in shards]
    assert max(loads) <= sum(loads) / 3 + max(n * m for n, m in zip(sizes, ms))
    assert shard.assign(sizes, ms, 1) == [list(range(len(sizes)))]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, sizes, ms, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    clouds = [cloudgen.uniform_cloud(n, seed=500 + b) for b, n in enumerate(sizes)]
    mine = shard.my_clouds(sizes, ms, world, rank)
    local = {b: oracle.fps(clouds[b], ms[b], 0).tolist() for b in mine}
    gathered = [None] * world
    dist.all_gather_object(gathered, local)
    if rank == 0:
        merged = {}
        for g in gathered:
            merged.update(g)
        q.put(merged)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_over_gloo_shard_without_collectives_on_data():
    sizes = [300, 1200, 700, 2000, 150, 900]
    ms = [max(1, n // 4) for n in sizes]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, sizes, ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert sorted(merged) == list(range(len(sizes)))
    for b, n in enumerate(sizes):
        assert merged[b] == oracle.fps(cloudgen.uniform_cloud(n, seed=500 + b), ms[b], 0).tolist()


def test_full_size_parity_covers_every_shape_the_bench_can_time():
    """The benchmark takes its launch shape and resolution from the library's two-stage autotuner;
    the full-size parity test runs every option set that tuner can return, and the space the bench
    line states is the tuner's."""
    import bench
    import test_gpu_fullsize
    from paper_2606_06255_gb300 import autotune
    assert bench.TUNER_SPACE == autotune.candidate_space(False)
    space = test_gpu_fullsize.tuner_space()
    for o in autotune.default_candidates(False):
        assert o in space
        for sc in autotune.NVOX_SCALES:
            assert (o if sc == 70 else dict(o, nvox_scale=sc)) in space


def test_reports_of_sharded_servers_merge_into_the_whole_stream():
    """Two servers (one per GPU) each serve half of a request stream; the merged report has every
    outcome once, the window and offered rate of the whole stream, and the same latencies."""
    reqs = _requests(40, rate=3000.0, seed=21)
    whole_window = (reqs[0].arrival, reqs[-1].arrival)
    parts = []
    for rank in range(2):
        clk = FakeClock()
        ex = SimExecutor(clk)
        mine = [r for r in reqs if r.rid % 2 == rank]
        parts.append(serve.Server(ex, mem_budget=10**9, max_inflight=3, max_batch=4).run(mine, clock=clk,
                                                                                      sleep=clk.sleep))
    merged = serve.merge_reports(parts)
    assert sorted(c.rid for c in merged.completed) == [r.rid for r in reqs]
    assert merged.window == whole_window
    assert abs(merged.offered_rate - (len(reqs) - 1) / (whole_window[1] - whole_window[0])) < 1e-9
    lat = sorted(c.latency for p in parts for c in p.completed)
    assert sorted(c.latency for c in merged.completed) == lat
    s = merged.summary()
    assert s["requests_completed"] == 40 and s["p99_latency_ms"] >= s["p50_latency_ms"] > 0
    assert s["samples_per_s"] > 0


class _FakeSmi:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _smi_line(mhz, power_cap="Not Active"):
    return f"0, {mhz}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, {power_cap}"


def test_clock_sampler_counts_only_the_timed_region_and_falls_back_to_adjacent_readings():
    import time
    import bench
    now = time.time()
    cs = bench.ClockSampler(0)
    cs.proc = _FakeSmi()
    cs.t0 = now - 1.0
    cs.lines = [(now - 2.0, _smi_line(1000)), (now - 0.5, _smi_line(2070)), (now - 0.4, _smi_line(2070, "Active"))]
    r = cs.stop()
    assert r["window"] == "timed" and r["samples"] == 2
    assert r["sm_mhz"] == 2070.0 and r["reasons"] == ["sw_power_cap"]
    # a timed region with no reading inside: the last one before it and the first one after it
    cs = bench.ClockSampler(0)
    cs.proc = _FakeSmi()
    cs.t0 = now - 0.01
    cs.lines = [(now - 3.0, _smi_line(500)), (now - 0.05, _smi_line(2060)), (now + 60.0, _smi_line(2070))]
    r = cs.stop()
    assert r["window"] == "adjacent" and r["samples"] == 2 and r["sm_mhz"] == 2065.0


def test_followups_continue_kept_sequences_exactly():
    """keep=True leaves a request's FPS state on the device; follow-ups (more_of) continue the
    same sequence: base + follow-ups equal one FPS run of the total M.  A follow-up that arrives
    while its base is still running waits for it; one of a request that was not kept fails; two
    follow-ups of the same state cannot both run (the second finds it moved on and fails)."""
    clk = FakeClock()
    ex = SimExecutor(clk, per_sample_s=1e-5)
    a = cloudgen.uniform_cloud(1500, seed=31)
    b = cloudgen.uniform_cloud(900, seed=32)
    reqs = [
        serve.Request(0, 0.0, a, 100, 7, keep=True),
        serve.Request(1, 0.0001, a, 50, 0, keep=True, more_of=0),   # arrives while 0 runs: waits
        serve.Request(2, 0.05, a, 25, 0, more_of=1),                 # the chain's last step: released
        serve.Request(3, 0.0, b, 40, 0),                             # not kept
        serve.Request(4, 0.05, b, 10, 0, more_of=3),                 # fails: nothing kept
        serve.Request(5, 0.0, b, 60, 2, keep=True),
        serve.Request(6, 0.06, b, 20, 0, more_of=5),
        serve.Request(7, 0.06, b, 20, 0, more_of=5),                 # same state as 6: fails
    ]
    rep = serve.Server(ex, mem_budget=10**7, max_inflight=4, max_batch=4).run(reqs, clock=clk, sleep=clk.sleep)
    by_id = {c.rid: c.indices for c in rep.completed}
    full_a = oracle.fps(a, 175, 7)
    np.testing.assert_array_equal(by_id[0], full_a[:100])
    np.testing.assert_array_equal(by_id[1], full_a[100:150])
    np.testing.assert_array_equal(by_id[2], full_a[150:175])
    np.testing.assert_array_equal(by_id[6], oracle.fps(b, 80, 2)[60:])
    assert sorted(rid for rid, _ in rep.failed) == [4, 7]
    assert rep.followups == 3
    # every kept state was released (consumed by a follow-up or at the end of the run)
    assert not ex.kept and sorted(ex.released) == [2, 6]
    assert [r for r in ex.launched if len(r) > 1 and {0, 1, 2, 5, 6} & set(r)] == []   # kept work runs alone


def test_followup_memory_is_held_until_released():
    """A kept index holds its bytes against the budget between its request and the follow-up."""
    clk = FakeClock()
    ex = SimExecutor(clk, bytes_per_point=1)
    ex.kept_size = 900_000
    a = cloudgen.uniform_cloud(1000, seed=33)
    others = [serve.Request(10 + i, 0.001 + 1e-4 * i, cloudgen.uniform_cloud(500, seed=40 + i), 50, 0)
              for i in range(6)]
    reqs = [serve.Request(0, 0.0, a, 100, 0, keep=True), serve.Request(1, 0.5, a, 100, 0, more_of=0)] + others
    rep = serve.Server(ex, mem_budget=1_000_000, max_inflight=4, max_batch=2).run(reqs, clock=clk, sleep=clk.sleep)
    assert len(rep.completed) == 8 and not rep.failed
    assert rep.peak_mem <= 1_000_000
    assert rep.peak_mem >= 900_000      # the kept index was counted while the others ran


class RoutingExecutor(SimExecutor):
    """Clouds of `tail_n` points or more run alone (as the GPU executor's size-aware route)."""

    def __init__(self, clock, tail_n, **kw):
        super().__init__(clock, **kw)
        self.tail_n = tail_n

    def alone(self, r):
        return r.points.shape[0] >= self.tail_n


def test_size_aware_routing_runs_large_clouds_alone():
    clk = FakeClock()
    ex = RoutingExecutor(clk, tail_n=1500)
    reqs = _requests(30, rate=5000.0, seed=8)
    rep = serve.Server(ex, mem_budget=10**8, max_inflight=4, max_batch=8).run(reqs, clock=clk, sleep=clk.sleep)
    assert len(rep.completed) == 30
    big = {r.rid for r in reqs if r.points.shape[0] >= 1500}
    assert big
    for b in ex.launched:
        if set(b) & big:
            assert len(b) == 1
    by_id = {c.rid: c.indices for c in rep.completed}
    for r in reqs:
        np.testing.assert_array_equal(by_id[r.rid], oracle.fps(r.points, r.m, r.start))


def test_bench_arms_print_the_same_config(capsys):
    """The reference arm (the CPU oracle) prints the same config dict as the GPU arm, which takes it
    from the same function, so the driver can pair the two lines."""
    import json

    import bench
    args = bench.parse(["--impl", "reference", "--workload", "uniform4k", "--steps", "1", "--warmup", "1"])
    assert bench.run_reference(args, 0) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "samples/s"
    assert line["config"] == bench.workload_config("uniform4k")[1]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_cpu_baseline_reports_the_three_oracle_timings():
    import bench
    c = bench.cpu_timing("uniform4k", budget_s=0.2)
    assert c["kind"] == "oracle" and c["value"] > 0 and c["cores"] >= 1
    assert c["plain_1thread"]["cores"] == 1 and c["plain_1thread"]["value"] > 0
    assert c["radiusfps_1thread"]["n_vox"] == 32 and c["radiusfps_1thread"]["value"] > 0


def test_batch_split_layout():
    """A size-split batch keeps each group's clouds contiguous (the tail group first) and maps every
    cloud back to its rows and output range in the caller's order."""
    from paper_2606_06255_gb300 import batch
    sizes = [5000, 120000, 800, 90000, 200000, 3000]
    ms = [s // 4 for s in sizes]
    bs = batch.BatchSampler(sizes, ms, opts={"cluster": 4}, device="cpu", graph=False,
                            split={"tail_n": 90000, "tail_opts": {"cluster": 16, "threads": 256}})
    assert [g.ids for g in bs.groups] == [[1, 3, 4], [0, 2, 5]]
    assert bs.groups[0].opts == {"cluster": 16, "threads": 256} and bs.groups[1].opts == {"cluster": 4}
    rows = sorted(bs.rows)
    assert rows[0][0] == 0 and rows[-1][1] == sum(sizes)
    assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))           # a partition of the buffer
    assert all(hi - lo == n for (lo, hi), n in zip(bs.rows, sizes))
    assert all(hi - lo == m for (lo, hi), m in zip(bs.out_rows, ms))
    assert max(bs.rows[i][1] for i in (1, 3, 4)) <= min(bs.rows[i][0] for i in (0, 2, 5))   # tail group first
    # three tiers: each cloud in the first tier it reaches, the largest tier first
    three = batch.BatchSampler(sizes, ms, opts={"cluster": 4}, device="cpu", graph=False,
                               split=[{"tail_n": 90000, "tail_opts": {"cluster": 8}},
                                      {"tail_n": 150000, "tail_opts": {"cluster": 16}}])
    assert [g.ids for g in three.groups] == [[4], [1, 3], [0, 2, 5]]
    assert [g.opts for g in three.groups] == [{"cluster": 16}, {"cluster": 8}, {"cluster": 4}]
    assert sorted(three.rows)[-1][1] == sum(sizes) and three.rows[4] == (0, 200000)
    # no split: one group in the caller's order
    one = batch.BatchSampler(sizes, ms, device="cpu", graph=False)
    assert len(one.groups) == 1 and one.rows[0] == (0, 5000) and one.rows[1] == (5000, 125000)


def test_batch_split_candidates():
    """The split tuner's candidates cut the batch between distinct sizes only, keep the k largest
    clouds in the tail group, and fall back to none for batches too small or too uniform to cut."""
    from paper_2606_06255_gb300 import autotune
    sizes = [1000 * (i + 1) for i in range(20)]            # 1k .. 20k, all distinct
    cands = autotune.split_candidates(sizes, {"cluster": 8})
    assert len(cands) == 3 * 2 * 2
    for rest, split in cands:
        tail = [n for n in sizes if n >= split["tail_n"]]
        assert len(tail) in (5, 8, 10)
        assert split["tail_opts"]["cluster"] in (8, 16) and rest["cluster"] in (4, 8)
    assert autotune.split_candidates([5000] * 20, None) == []          # no size to cut between
    assert autotune.split_candidates([300, 200, 100], None) == []      # fewer clouds than any k
    tied = [20] * 4 + [10] * 4 + [5] * 12     # only the 8 largest separate cleanly from the rest
    got = autotune.split_candidates(tied, None)
    assert got and {len([n for n in tied if n >= s["tail_n"]]) for _, s in got} == {8}
