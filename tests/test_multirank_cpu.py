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
