"""The multi-rank logic of bench.py on CPU: two gloo ranks (127.0.0.1), each with its own
time; the job's time is the slowest rank's and its throughput counts every rank's
replica of the workload (weak scaling, no data-path collective)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = 1.0 + rank  # rank 1 is slower
    tmax = bench.max_over_ranks(t, dist, "cpu")
    v = bench.job_throughput(1000, world, 4, tmax)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, tmax, v))


def test_two_gloo_ranks_max_time_and_weak_scaling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, tmax, v in res:
        assert tmax == 2.0                    # the slowest rank's time on both ranks
        assert v == pytest.approx(1000 * 2 * 4 / 2.0)  # both replicas' units over that time


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_throughput(10, 1, 2, 4.0) == 5.0


def test_oracle_all_cores_runs_and_counts_points():
    """The all-cores oracle baseline: one spawned process per window, all points counted."""
    import bench
    from oracle import marfa_oracle as O
    from workloads import config0_tiny
    wl = config0_tiny()
    v, pts, dt = bench.oracle_all_cores(wl, 0, 4000.0, 0.03125, 2)
    assert pts == 2 * O.num_points(4000.0, 4000.03125) and dt > 0 and v == pts / dt


def test_reference_arm_line_on_a_small_workload():
    """`bench.py --impl reference` prints the contract's JSON line (the oracle on every
    host core), here on the small one-level workload."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload",
                        "tiny", "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "pts*levels/s"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["cores"] >= 1


# ------------------------------------------------------------ level-sharded jobs
def test_level_shards_cover_each_level_once():
    from paper_2411_03418_gb300.shard import level_shards, request_shards
    rng = __import__("numpy").random.default_rng(3)
    for n in (1, 5, 60, 61):
        for world in (1, 2, 3, 8):
            cost = rng.uniform(1.0, 10.0, n)
            for mode in ("interleaved", "contiguous", "balanced"):
                sh = level_shards(n, world, cost=cost, mode=mode)
                assert len(sh) == world
                flat = sorted(x for s in sh for x in s)
                assert flat == list(range(n)), (n, world, mode)
                assert all(s == sorted(s) for s in sh)
            # contiguous blocks differ in size by at most one level
            sizes = [len(s) for s in level_shards(n, world, mode="contiguous")]
            assert max(sizes) - min(sizes) <= 1
            # balanced: no rank above the mean cost plus one level's cost
            sh = level_shards(n, world, cost=cost, mode="balanced")
            loads = [cost[s].sum() for s in sh]
            assert max(loads) <= cost.sum() / world + cost.max() + 1e-9
    assert request_shards(7, 3) == [[0, 3, 6], [1, 4], [2, 5]]
    with pytest.raises(ValueError):
        level_shards(4, 0)


def _shard_rank(rank, world, port, q):
    """One gloo rank of a level-split job: the FP64 oracle stands in for the GPU call on
    this rank's levels of a small multi-level workload; the blocks are gathered on rank 0."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np
    import torch
    from oracle import marfa_oracle as O
    from paper_2411_03418_gb300.shard import gather_levels, level_shards
    from workloads import tiny_workload
    wl = tiny_workload(91, 60, 2000.0, 2000.25, 10.0, T=(700.0, 500.0, 300.0, 200.0, 170.0),
                       p=(50.0, 5.0, 0.5, 0.01, 1e-4), chi="tonkov", chi_species=1)
    mine = level_shards(wl.n_levels, world, mode="contiguous")[rank]
    block = torch.from_numpy(np.stack([O.eleven_grid(wl, lev) for lev in mine]) if mine
                             else np.zeros((0, O.num_points(wl.nu_lo, wl.nu_hi))))
    full = gather_levels(block, mine, wl.n_levels, dist, dst=0)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, None if full is None else full.numpy()))


def test_level_split_over_gloo_ranks_equals_one_rank():
    """Three gloo ranks split five levels (2 + 2 + 1) and gather them on rank 0: the
    joined array equals the single-rank result level for level, bit for bit."""
    import numpy as np
    from oracle import marfa_oracle as O
    from workloads import tiny_workload
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 3
    procs = [ctx.Process(target=_shard_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert res[1] is None and res[2] is None
    wl = tiny_workload(91, 60, 2000.0, 2000.25, 10.0, T=(700.0, 500.0, 300.0, 200.0, 170.0),
                       p=(50.0, 5.0, 0.5, 0.01, 1e-4), chi="tonkov", chi_species=1)
    ref = np.stack([O.eleven_grid(wl, lev) for lev in range(wl.n_levels)])
    assert res[0].shape == ref.shape and np.array_equal(res[0], ref)


def test_gather_levels_on_one_rank_reorders():
    import torch
    from paper_2411_03418_gb300.shard import gather_levels
    blk = torch.arange(12, dtype=torch.float32).reshape(3, 4)
    out = gather_levels(blk, [2, 0, 1], 3, None)
    assert torch.equal(out[2], blk[0]) and torch.equal(out[0], blk[1]) and torch.equal(out[1], blk[2])
