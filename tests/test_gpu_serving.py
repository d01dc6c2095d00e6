"""Batching, CUDA-graph replay, autotuning and serving on the GPU."""

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


def _mixed(n, seed):
    rng = np.random.default_rng(seed)
    clouds = []
    for b in range(n):
        size = int(rng.integers(3000, 40000))
        pts = cloudgen.room_cloud(size, seed=seed + b) if b % 2 == 0 else cloudgen.lidar_cloud(size, seed=seed + b)
        clouds.append(pts)
    return clouds


def test_serving_results_identical_alone_and_in_the_mix(rf):
    clouds = _mixed(14, 700)
    rng = np.random.default_rng(1)
    t = np.cumsum(rng.exponential(1.0 / 2000.0, size=len(clouds)))
    reqs = [rf.serve.Request(i, float(t[i]), c, max(1, c.shape[0] // 8), i % 5) for i, c in enumerate(clouds)]
    ex = rf.serve.GpuExecutor(n_slots=3, opts={"cluster": 4})
    rep = rf.serve.Server(ex, mem_budget=1 << 30, max_inflight=3, max_batch=4).run(reqs)
    assert len(rep.completed) == len(reqs) and not rep.rejected
    by_id = {c.rid: c for c in rep.completed}
    for r in reqs:
        alone = rf.fps(torch.from_numpy(r.points).cuda(), r.m, r.start, check=True).cpu().numpy()
        np.testing.assert_array_equal(by_id[r.rid].indices, alone)
        np.testing.assert_array_equal(alone, oracle.fps(r.points, r.m, r.start, threads=0))
    s = rep.summary()
    assert s["p99_latency_ms"] >= s["p50_latency_ms"] > 0
    assert rep.max_inflight_batches >= 2      # batches overlapped on the device


def test_graph_replayed_batch(rf):
    clouds = _mixed(6, 900)
    sizes = [c.shape[0] for c in clouds]
    ms = [n // 4 for n in sizes]
    bs = rf.batch.BatchSampler(sizes, ms, opts={"cluster": 2})
    bs.load(clouds)
    out1 = bs.split(bs.run().clone())
    out2 = bs.split(bs.run())
    assert bs.status() == 0
    for b, c in enumerate(clouds):
        ref = oracle.fps(c, ms[b], 0, threads=0)
        np.testing.assert_array_equal(out1[b], ref)
        np.testing.assert_array_equal(out2[b], ref)
    # a new batch of the same shape through the same graph
    other = [cloudgen.uniform_cloud(n, seed=77 + i) for i, n in enumerate(sizes)]
    bs.load(other)
    out3 = bs.split(bs.run())
    for b, c in enumerate(other):
        np.testing.assert_array_equal(out3[b], oracle.fps(c, ms[b], 0, threads=0))


@pytest.mark.parametrize("split", [{"tail_n": 40000, "tail_opts": {"cluster": 8, "threads": 256}},
                                   {"tail_n": 40000, "tail_opts": {"cluster": 16, "threads": 128, "chunk": 64}},
                                   [{"tail_n": 50000, "tail_opts": {"cluster": 16, "threads": 256}},
                                    {"tail_n": 40000, "tail_opts": {"cluster": 8, "threads": 256}}]],
                         ids=["two_8", "two_16", "three_tiers"])
def test_graph_replayed_split_batch(rf, split):
    """The largest clouds in concurrent launches of their own (BatchSampler's size split, in two or
    three tiers), all launches in one graph: every cloud's indices are the oracle's, in the caller's
    order, on two replays, and the same as the unsplit batch's."""
    clouds = _mixed(8, 1200) + [cloudgen.lidar_cloud(60000, seed=91), cloudgen.room_cloud(45000, seed=92)]
    sizes = [c.shape[0] for c in clouds]
    ms = [n // 6 for n in sizes]
    bs = rf.batch.BatchSampler(sizes, ms, opts={"cluster": 2, "threads": 256}, split=split)
    assert len(bs.groups) == (3 if isinstance(split, list) else 2)
    assert sorted(i for g in bs.groups[:-1] for i in g.ids) == [8, 9]
    bs.load(clouds)
    out1 = bs.split(bs.run().clone())
    out2 = bs.split(bs.run())
    assert bs.status() == 0
    plain = rf.batch.BatchSampler(sizes, ms, opts={"cluster": 2, "threads": 256})
    plain.load(clouds)
    out3 = plain.split(plain.run())
    for b, c in enumerate(clouds):
        ref = oracle.fps(c, ms[b], 0, threads=0)
        np.testing.assert_array_equal(out1[b], ref)
        np.testing.assert_array_equal(out2[b], ref)
        np.testing.assert_array_equal(out3[b], ref)


def test_autotune_picks_a_candidate_with_identical_results(rf, tmp_path):
    pts_np = cloudgen.room_cloud(20000, seed=5)
    pts = torch.from_numpy(pts_np).cuda()
    cands = [{"cluster": 2, "threads": 256}, {"cluster": 8, "threads": 256, "chunk": 64}]
    best, table = rf.autotune.tune_single(pts, 4000, 0, candidates=cands, reps=1, scales=(50, 100))
    space = cands + [dict(c, nvox_scale=s) for c in cands for s in (50, 100)]
    assert best in space and len(table) == 6 and sorted(map(str, (o for _, o in table))) == sorted(map(str, space))
    path = str(tmp_path / "tune.json")
    rf.autotune.save(rf.autotune.key("room", 20000), best, table, path=path)
    assert rf.autotune.best_opts("room", 20000, path=path) == best
    got = rf.fps(pts, 4000, 0, opts=best, check=True).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.fps(pts_np, 4000, 0, threads=0))


def test_device_error_fails_only_the_bad_request(rf):
    """A cloud with a non-finite coordinate makes its micro-batch report RFPS_ENONFINITE on the device:
    the server reruns that batch's clouds one by one, serves the others and reports the bad one."""
    clouds = _mixed(6, 1300)
    bad = clouds[2].copy()
    bad[17, 1] = np.nan
    clouds[2] = bad
    reqs = [rf.serve.Request(i, 0.0, c, max(1, c.shape[0] // 16), 0) for i, c in enumerate(clouds)]
    ex = rf.serve.GpuExecutor(n_slots=2, opts={"cluster": 2})
    rep = rf.serve.Server(ex, mem_budget=1 << 30, max_inflight=2, max_batch=6, max_retries=1).run(reqs)
    assert [rid for rid, _ in rep.failed] == [2]
    assert "device status" in rep.failed[0][1]
    by_id = {c.rid: c for c in rep.completed}
    assert sorted(by_id) == [0, 1, 3, 4, 5]
    for r in reqs:
        if r.rid in by_id:
            np.testing.assert_array_equal(by_id[r.rid].indices, oracle.fps(r.points, r.m, r.start, threads=0))


def test_serving_launch_shape_at_full_size(rf):
    """The serving benchmark's launch shape (one 512-thread CTA per cloud, records beyond shared
    memory on the hierarchical path) on a micro-batch holding the largest clouds its request stream
    draws: the full 1.12M-point LiDAR scan and a 1M-point room, with M = N/8, next to two small
    clouds; every cloud's indices against the oracle, element by element."""
    clouds = [cloudgen.lidar_cloud(None, seed=0), cloudgen.room_cloud(1_000_000, seed=91),
              cloudgen.room_cloud(20_000, seed=92), cloudgen.lidar_cloud(50_000, seed=93, scan_seed=1)]
    sizes = [c.shape[0] for c in clouds]
    ms = [n // 8 for n in sizes]
    starts = [0, 17, 3, 49_999]
    cat = torch.from_numpy(np.concatenate(clouds)).cuda()
    refs = [oracle.fps(c, ms[b], starts[b], threads=0) for b, c in enumerate(clouds)]
    opts = {"cluster": 1, "threads": 512}
    ws = torch.empty(rf.batch_workspace_size(cat.shape[0], len(clouds), max(sizes), opts), dtype=torch.uint8,
                     device="cuda")
    out, ooff = rf.fps_batched(cat, sizes, ms, starts, opts=opts, workspace=ws)
    assert rf.status(ws) == 0
    out = out.cpu().numpy()
    for b, c in enumerate(clouds):
        np.testing.assert_array_equal(out[ooff[b]:ooff[b + 1]], refs[b], err_msg=f"cloud {b} (N={sizes[b]})")
    # the serving benchmark's size-aware route: each large cloud alone on an 8-CTA cluster
    import bench
    for b in range(2):
        got = rf.fps_batched(torch.from_numpy(clouds[b]).cuda(), [sizes[b]], [ms[b]], [starts[b]],
                             opts=bench.TAIL_OPTS)[0].cpu().numpy()
        np.testing.assert_array_equal(got, refs[b], err_msg=f"routed cloud {b} (N={sizes[b]}), {bench.TAIL_OPTS}")
    assert sizes[0] >= bench.TAIL_N and sizes[1] >= bench.TAIL_N


def test_followups_on_kept_indices_and_tail_routing(rf):
    """Follow-up requests continue a kept device index (rfps_index_sample_more): each piece equals
    the matching slice of one oracle run of the total M.  Clouds above tail_n points run alone with
    the tail launch shape; everything served equals the oracle."""
    a = cloudgen.room_cloud(30000, seed=95)
    b = cloudgen.lidar_cloud(60000, seed=96)
    small = [cloudgen.room_cloud(int(n), seed=97 + i) for i, n in enumerate((4000, 9000, 7000))]
    reqs = [rf.serve.Request(0, 0.0, a, 1000, 5, keep=True),
            rf.serve.Request(1, 0.0005, a, 2000, 0, keep=True, more_of=0),
            rf.serve.Request(2, 0.002, a, 500, 0, more_of=1),
            rf.serve.Request(3, 0.0, b, 6000, 11),                       # tail route (N >= 50,000)
            ] + [rf.serve.Request(4 + i, 0.0001 * i, c, c.shape[0] // 8, 0) for i, c in enumerate(small)]
    ex = rf.serve.GpuExecutor(n_slots=3, opts={"cluster": 1, "threads": 512},
                              tail_opts={"cluster": 4, "threads": 256}, tail_n=50000)
    rep = rf.serve.Server(ex, mem_budget=1 << 30, max_inflight=3, max_batch=4).run(reqs)
    assert not rep.failed and len(rep.completed) == len(reqs)
    assert rep.followups == 2 and not ex.kept        # chain consumed, nothing left on the device
    by_id = {c.rid: c for c in rep.completed}
    full_a = oracle.fps(a, 3500, 5, threads=0)
    np.testing.assert_array_equal(by_id[0].indices, full_a[:1000])
    np.testing.assert_array_equal(by_id[1].indices, full_a[1000:3000])
    np.testing.assert_array_equal(by_id[2].indices, full_a[3000:])
    np.testing.assert_array_equal(by_id[3].indices, oracle.fps(b, 6000, 11, threads=0))
    assert by_id[3].batch_size == 1
    for i, c in enumerate(small):
        np.testing.assert_array_equal(by_id[4 + i].indices, oracle.fps(c, c.shape[0] // 8, 0, threads=0))
