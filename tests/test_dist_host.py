"""The multi-rank host logic of bench.py on CPU: two gloo ranks (one replica each) agree
on the slowest rank's time, the whole-job rate counts every rank's units, the batch of
128 graphs is split over the ranks by cost with every graph rendered exactly once, and
the reference arm runs on rank 0 only.  No GPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [3.0, 5.0][rank]                       # rank 1 is the slow one
        dist.barrier()
        t = bench.max_over_ranks(ms, dist, "cpu")
        q.put((rank, t, bench.job_rate(1000, world, 4, t)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_the_job_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[1] for g in got] == [5.0, 5.0]
    # 1000 units per rank and step, 2 ranks, 4 steps in 5 ms
    assert all(abs(g[2] - 1000 * 2 * 4 / 5e-3) < 1e-6 for g in got)


def _shard_rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    from paper_2408_03204_b300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        graphs, lengths, _ = bench.workload("batch128")
        costs = [g.n_nodes * L for g, L in zip(graphs, lengths)]
        mine = shard.partition(costs, world)[rank]          # no exchange needed to agree
        P = bench.params_for("batch128", graphs, "param")
        rows = shard.rows_of(graphs, mine, P)
        got = [None] * world
        dist.all_gather_object(got, (mine, {t: v.shape for t, v in rows.items()}))
        q.put((rank, got, sum(costs[k] for k in mine)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_batch_by_graph():
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import bench
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got[0][1] == got[1][1]                       # both ranks see the same split
    parts = [m for m, _ in got[0][1]]
    assert sorted(parts[0] + parts[1]) == list(range(128))   # every graph exactly once
    graphs, lengths, _ = bench.workload("batch128")
    costs = [g.n_nodes * L for g, L in zip(graphs, lengths)]
    loads = [c for _, _, c in got]
    assert max(loads) <= sum(costs) / 2 + max(costs)    # list-scheduling bound
    assert max(loads) <= 1.01 * sum(costs) / 2          # and close to even on this batch
    # each rank's parameter tables hold exactly its graphs' rows
    for (mine, shapes) in got[0][1]:
        for t, shp in shapes.items():
            assert shp[0] == sum(graphs[k].count(t) for k in mine)


def test_partition_properties():
    from paper_2408_03204_b300 import shard
    import random
    rng = random.Random(5)
    for world in (1, 2, 3, 8):
        costs = [rng.randint(1, 1000) for _ in range(rng.randint(0, 40))]
        parts = shard.partition(costs, world)
        assert len(parts) == world and sorted(sum(parts, [])) == list(range(len(costs)))
        assert all(p == sorted(p) for p in parts)
        assert parts == shard.partition(costs, world)    # deterministic
        if costs:
            loads = [sum(costs[k] for k in p) for p in parts]
            assert max(loads) <= sum(costs) / world + max(costs)


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, None, "cpu") == 2.5
    assert bench.job_rate(10, 1, 2, 4.0) == 10 * 2 / 4e-3


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the reference arm prints on rank 0; other ranks exit 0 silently."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--ref-sample", "2"], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["config"]["same_config"] and line["cpu_baseline"]["cores"] == 2
