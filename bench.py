"""Throughput of the eleven-grid line-by-line path on the Venus workload.

Workload: 200,000 band-structured CO2-like lines over 1875-3125 cm^-1, 60 Venus
levels (735 -> 170 K, 92 -> 1e-5 atm), Voigt x Tonkov chi-factor, 125 cm^-1 cut-off,
k(nu) on 2000-3000 cm^-1 at 2^-11 cm^-1 (2,048,001 points per level). One step =
one replay of the request's captured plan (marfa_plan_execute: level preparation,
grid 1, grids 2..10 with their autotuned kernels, finest grid with the interpolation
cascade, over all 60 levels) with the line list resident on the GPU.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload venus|batch|earth|tiny]

The default (and headline) workload is the Venus one; --workload times the other
configurations the same way (batch: 256 uneven requests in one plan; earth: 1.2M lines
x 50 levels; tiny: 2,000 lines x 1 level).

Prints one JSON line. ``value`` is fine-grid points x levels per second over all
ranks (with N > 1 ranks the levels, or a batch's requests, are split over them:
strong scaling, no data-path collective); ``line_evals_per_s`` counts the (line, node) profile evaluations the scheme
defines. ``e2e`` is the same metric through the public call with host buffers
(line records and levels from pinned host memory in, k(nu) back to pinned host
memory, every step). ``--impl reference`` times the FP64 CPU oracle on a bounded
sample of the same workload (there is no other implementation of this path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import queue
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spectral pts x levels/s and line-evals/s, MLP-Voigt vs plain at <=1e-3 rel err"
UNIT = "pts*levels/s"
# FP32 flops of one profile evaluation by Voigt cost class, counted from the formulas
# (x, the profile, amplitude, chi-factor and the compensated add): far-wing two-term
# series, 6/15-term asymptotic series (the 6-term count is used for both), 9 x 9
# polynomial cell plus the Gaussian term, small-y cell (6 x 4 terms) plus the Gaussian term.
FLOPS_FAR, FLOPS_MID, FLOPS_NEAR, FLOPS_SMALL = 20.0, 70.0, 200.0, 90.0

# DRAM bytes (read + write) per launch of the dominant kernel of the Venus workload's
# full window, by the variant the plan chose, from a single-pass ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum; command and figures in
# profiles/traffic_dominant_kernels.md). Finest-grid variants: 1 flattened jobs, 2 the
# same by mechanism, 3 by mechanism merged. They belong to the kernels as built when
# captured; other workloads, windows and variants report null.
TRAFFIC_BYTES = {("venus", "finest", 1): 653.5e6 + 620.3e6,
                 ("venus", "finest", 2): 642.0e6 + 459.9e6,
                 ("venus", "finest", 3): 642.9e6 + 465.0e6}
N_SM = 152
FP32_LANES = 128


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("sm_max_mhz", 2070.0), "measured"
    return 2070.0, "fallback"


def start_clock_sampler(path):
    try:
        f = open(path, "w")
        return subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
             "--format=csv,noheader,nounits", "-lms", "50"], stdout=f, stderr=subprocess.DEVNULL), f
    except (OSError, FileNotFoundError):
        return None, None


def sampler_lines(path, wait_s=0.0):
    """Lines the clock sampler has written so far; with wait_s, first wait (at most that
    long) until it has written one, so that the timed region starts with the sampler
    running."""
    t_end = time.perf_counter() + wait_s
    while True:
        try:
            with open(path) as f:
                n = sum(1 for _ in f)
        except OSError:
            n = 0
        if n > 0 or time.perf_counter() >= t_end:
            return n
        time.sleep(0.01)


def read_clocks(path, dev_index, skip=0):
    """Median SM clock, max clock and throttle reasons of the sampler's rows for this
    device, leaving out the first `skip` lines (written before the timed region) when
    rows remain after them."""
    rows = []
    try:
        for k, line in enumerate(open(path)):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9 and parts[0] == str(dev_index):
                rows.append((k, parts))
    except OSError:
        return None
    if any(k >= skip for k, _ in rows):
        rows = [r for r in rows if r[0] >= skip]
    rows = [r for _, r in rows]
    if not rows:
        return None
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
    return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": reasons,
            "samples": len(rows)}


def _oracle_sample(wl, lev, lo, hi):
    """The workload cut to one level, the window [lo, hi] and the lines that can reach it
    (the others contribute nothing)."""
    keep = np.abs(wl.lines["nu0"] - 0.5 * (lo + hi)) <= wl.cutoff + 2.0
    return wl.with_(lines=wl.lines[keep], nu_lo=lo, nu_hi=hi).level_subset([lev]), int(keep.sum())


def _sample_place(wl, width, count):
    """The middle level of the workload and the start (a multiple of 2^-11 cm^-1) of
    `count` adjacent windows of `width` cm^-1 centred in its window (Venus: level 30 of 60,
    16 windows of 0.125 cm^-1 from 2499 cm^-1)."""
    lev = wl.n_levels // 2
    lo = 0.5 * (wl.nu_lo + wl.nu_hi) - 0.5 * width * count
    lo = max(wl.nu_lo, min(lo, wl.nu_hi - width * count))
    return lev, math.floor(lo * 2048.0) / 2048.0


def _oracle_worker(sub, barrier, q):
    """One process of the all-cores oracle run (spawn start): waits for the others, then
    runs the eleven-grid oracle on its sample and reports its start and end times."""
    from oracle import marfa_oracle as O
    barrier.wait(timeout=600.0)
    t0 = time.monotonic()
    O.eleven_grid(sub, 0)
    q.put((t0, time.monotonic()))


def oracle_all_cores(wl, lev, lo, width, nproc):
    """The FP64 oracle (as it stands) on nproc adjacent windows of the given width at one
    level, one process per host core, all started together: (points per second over the
    whole run, points, seconds)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    barrier, q = ctx.Barrier(nproc), ctx.Queue()
    subs = [_oracle_sample(wl, lev, lo + i * width, lo + (i + 1) * width)[0] for i in range(nproc)]
    procs = [ctx.Process(target=_oracle_worker, args=(s, barrier, q)) for s in subs]
    for p in procs:
        p.start()
    spans, deadline = [], time.monotonic() + 900.0
    try:
        while len(spans) < nproc:
            try:
                spans.append(q.get(timeout=1.0))
            except queue.Empty:
                if any(p.exitcode not in (None, 0) for p in procs) or time.monotonic() > deadline:
                    raise RuntimeError("an oracle worker process failed or timed out")
    finally:
        for p in procs:
            p.join(timeout=30.0)
            if p.is_alive():
                p.kill()
    from oracle import marfa_oracle as O
    pts = sum(O.num_points(s.nu_lo, s.nu_hi) for s in subs)
    dt = max(b for _, b in spans) - min(a for a, _ in spans)
    return pts / dt, pts, dt


def cpu_baseline_sample(wl):
    """Time the FP64 oracle (as it stands) on a bounded sample of the workload: the
    eleven-grid result of one mid-profile level on windows of 0.25 cm^-1, once on one
    core and then on every host core at once (one window per process)."""
    from oracle import marfa_oracle as O
    width = 0.25
    nproc = os.cpu_count() or 1
    lev, lo = _sample_place(wl, width, nproc)
    sub, nin = _oracle_sample(wl, lev, lo, lo + width)
    t = time.perf_counter()
    O.eleven_grid(sub, 0)
    dt1 = time.perf_counter() - t
    pts1 = O.num_points(lo, lo + width)
    v, pts, dt = oracle_all_cores(wl, lev, lo, width, nproc)
    return {"value": v, "unit": UNIT, "cores": nproc, "kind": "oracle",
            "single_core_value": pts1 / dt1,
            "sample": f"level {lev}, {nproc} adjacent windows of {width} cm^-1 from {lo} cm^-1 "
                      f"({pts} points, one process per core, {dt:.1f} s); single core: {lo}-{lo + width} "
                      f"cm^-1 ({pts1} points, {nin} lines in reach, {dt1:.1f} s); numpy/scipy FP64"}


def run_reference(args, wl, rank, world):
    if rank != 0:
        return
    nproc = os.cpu_count() or 1
    width = 0.125
    lev, lo = _sample_place(wl, width, nproc)
    times, pts = [], 0
    for i in range(args.warmup + args.steps):
        _, pts, dt = oracle_all_cores(wl, lev, lo, width, nproc)
        if i >= args.warmup:
            times.append(dt)
    dt = float(np.mean(times))
    v = pts / dt
    sample = (f"level {lev}, {nproc} adjacent windows of {width} cm^-1 from {lo} cm^-1 per step "
              f"({pts} points, one process per core)")
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": nproc, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def surrogate_leg(args, M, wl, lines, levels, out, flush, stream, wpath, evals_plain, ms_plain, npts, dist,
                  dev):
    """The same workload with the learned Voigt under its guard: throughput, the share
    of evaluations the surrogate took, and its largest relative deviation from the
    plain FP32 path (both outputs on the device, compared where k > 1e-8 of the level's
    maximum)."""
    import torch
    budget, lattice = 6e-4, 32
    on, _ = M.marfa_surrogate_load(np.load(wpath).astype(np.float32), budget, lattice)
    try:
        plain = out.clone()
        rq_s = M.request_of(wl.with_(surrogate=1))
        if args.no_count:
            c5 = np.zeros((wl.n_levels, 11, 5), dtype=np.int64)
        else:
            _, c5 = M.marfa_diag_absorption_counts(lines, levels, wl.vmr, rq_s)
        counts, sc = c5[:, :, 0], c5[:, :, 1]
        plan = M.marfa_plan_create([lines], [levels], [wl.vmr], [rq_s], [out], autotune=True, stream=stream)
        for _ in range(args.warmup):
            M.marfa_plan_execute(plan, stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            M.marfa_plan_execute(plan, stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        kms_s = M.marfa_plan_info(plan, kernel_ms=True)[2]
        M.marfa_plan_destroy(plan)
        t_total = max_over_ranks(float(sum(a.elapsed_time(b) for a, b in ev)) / 1e3, dist, dev)
        world = dist.get_world_size() if dist else 1
        mx = plain.abs().amax(dim=1, keepdim=True)
        big = plain.abs() > 1e-8 * mx
        rel = ((out - plain).abs() / plain.abs().clamp_min(1e-38))[big]
        ms = t_total / args.steps * 1e3
        return {"value": job_throughput(wl.n_levels * npts, world, args.steps, t_total), "unit": UNIT,
                "ms_per_step": ms,
                "line_evals_per_s": job_throughput(int(counts.sum()), world, args.steps, t_total),
                "surrogate_evals_share": float(sc.sum() / max(1, counts.sum())),
                "surrogate_evals_per_grid": [int(v) for v in sc.sum(axis=0)],
                "kernel_ms_last_step": [round(float(v), 3) for v in kms_s],
                "max_rel_vs_plain": float(rel.max().item()), "guard_budget": budget, "guard_lattice": lattice, "guard_cells_on": int(on),
                "speedup_vs_plain": ms_plain / ms,
                "note": "plain path within 1e-4 of the FP64 oracle; surrogate path within 1e-3 (tests)"}
    finally:
        M.marfa_surrogate_unload()


def max_over_ranks(t, dist, dev):
    """The largest of the ranks' values of t (a float), or t itself on one rank."""
    if not dist:
        return float(t)
    import torch
    tt = torch.tensor([float(t)], dtype=torch.float64, device=dev)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def marfa_points(w):
    """Finest-grid nodes of a workload's window (k 2^-11 in [nu_lo, nu_hi])."""
    return int(math.floor(w.nu_hi * 2048.0) - math.ceil(w.nu_lo * 2048.0) + 1)


def sum_over_ranks(x, dist, dev):
    """The sum of the ranks' values of x (an integer), or x itself on one rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([int(x)], dtype=torch.int64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return int(t.item())


def job_throughput(units_per_rank, world, steps, t_max):
    """Whole-job rate over the slowest rank's time: world x units x steps / t_max, where
    each of `world` ranks processes `units_per_rank` per step (a replica per rank, weak
    scaling; for a job split over the ranks pass the job's units and world = 1)."""
    return units_per_rank * world * steps / t_max


def load_workloads(name):
    from workloads import config0_tiny, config1_venus, config2_batch, config3_earth
    if name == "venus":
        return [config1_venus()], "venus"
    if name == "batch":
        return config2_batch(), "batch: 256 uneven requests (1-50 cm-1 windows in 500-5000, 1k-50k lines, " \
                                "1-100 Venus levels, cut-off 25/125)"
    if name == "earth":
        return [config3_earth()], None
    return [config0_tiny()], None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["venus", "batch", "earth", "tiny"], default="venus",
                    help="venus (default, the headline), or a parity configuration timed the same way")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nu-lo", type=float, default=None, help="narrow the window (profiling runs)")
    ap.add_argument("--nu-hi", type=float, default=None)
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer steps")
    ap.add_argument("--no-count", action="store_true", help="skip the evaluation-counting call")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the learned-Voigt leg")
    ap.add_argument("--shard", choices=["auto", "levels", "requests", "none"], default="auto",
                    help="with N > 1 ranks: split the levels (one request) or the requests (a batch) "
                         "over the ranks (strong scaling; auto), or run a replica per rank (none)")
    ap.add_argument("--stencil", type=int, choices=[3, 5], default=3,
                    help="interpolation points per coarse panel: 3 (the paper's) or 5 (quartic)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    wls, wname = load_workloads(args.workload)
    if args.stencil != 3:
        wls = [w.with_(stencil=args.stencil) for w in wls]
    if args.nu_lo is not None or args.nu_hi is not None:
        wls = [w.with_(nu_lo=args.nu_lo if args.nu_lo is not None else w.nu_lo,
                       nu_hi=args.nu_hi if args.nu_hi is not None else w.nu_hi) for w in wls]
    wl = wls[0]
    wname = wname or wl.name
    if wname == "venus":
        wname = wl.name

    if args.impl == "reference":
        run_reference(args, wl, rank, world)
        return

    # the whole job's work, then this rank's share of it (levels are independent, and so
    # are the requests of a batch: no exchange step between the ranks)
    units_job = sum(w.n_levels * marfa_points(w) for w in wls)
    shard = args.shard
    if shard == "auto":
        shard = "none" if world == 1 else ("levels" if len(wls) == 1 else "requests")
    if world > 1 and shard != "none":
        from paper_2411_03418_gb300.shard import level_shards, request_shards
        if shard == "levels":
            if any(w.n_levels < world for w in wls):
                raise SystemExit("fewer levels than ranks: use --shard requests or none")
            wls = [w.level_subset(level_shards(w.n_levels, world)[rank]) for w in wls]
        else:
            if len(wls) < world:
                raise SystemExit("fewer requests than ranks: use --shard levels or none")
            wls = [wls[i] for i in request_shards(len(wls), world)[rank]]
    else:
        units_job *= world  # a replica of the workload per rank

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    import __graft_entry__
    if rank == 0 or not dist:
        __graft_entry__.build()  # one rank compiles (if needed); the others wait
    if dist:
        dist.barrier()
        __graft_entry__.build()  # finds the library up to date
    from paper_2411_03418_gb300 import marfa as M

    stream = torch.cuda.current_stream()
    lines = [M.marfa_prepare_lines(w.lines, w.species) for w in wls]
    levels = [M.levels_of(w) for w in wls]
    rqs = [M.request_of(w) for w in wls]
    npts = [M.marfa_num_points(w.nu_lo, w.nu_hi) for w in wls]
    outs = [torch.empty((w.n_levels, n), dtype=torch.float32, device=dev) for w, n in zip(wls, npts)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

    # evaluation counts of one step (exact, from the counting variant of the kernels)
    c5 = np.zeros((11, 5), dtype=np.int64)
    if not args.no_count:
        for q, w in enumerate(wls):
            c5 += M.marfa_diag_absorption_counts(lines[q], levels[q], w.vmr, rqs[q])[1].sum(axis=0)
    counts_grid = c5[:, 0]
    evals_per_step = int(counts_grid.sum())
    # algorithmic flops per grid by Voigt cost class
    n_near, n_mid, n_small = c5[:, 2], c5[:, 3], c5[:, 4]
    n_far = counts_grid - n_near - n_mid - n_small
    flops_grid = FLOPS_FAR * n_far + FLOPS_MID * n_mid + FLOPS_NEAR * n_near + FLOPS_SMALL * n_small

    t0 = time.perf_counter()
    plan = M.marfa_plan_create(lines, levels, [w.vmr for w in wls], rqs, outs, autotune=True, stream=stream)
    plan_s_create = time.perf_counter() - t0
    variant, tune_ms, _ = M.marfa_plan_info(plan)
    req_class, class_choice, _ = M.marfa_plan_classes(plan, len(wls))

    def step():
        M.marfa_plan_execute(plan, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()

    clk_path = os.path.join(tempfile.gettempdir(), f"marfa_clocks_{os.getpid()}.csv")
    sampler, fh = start_clock_sampler(clk_path)
    n_before = sampler_lines(clk_path, 5.0) if sampler else 0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(float(i))  # L2 flush between steps, outside the timed events
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    klaunch = np.full(12, args.steps, dtype=np.int64)  # one launch of each kind per step
    step_ms = [a.elapsed_time(b) for a, b in ev]
    if sampler:
        sampler.terminate()
        sampler.wait()
        fh.close()
    clocks = read_clocks(clk_path, torch.cuda.current_device(), n_before) if sampler else None
    t_total = max_over_ranks(float(sum(step_ms)) / 1e3, dist, dev)
    ms_per_step = t_total / args.steps * 1e3
    M.marfa_plan_destroy(plan)
    # per-kernel times for the roofline: the same work as a serial plan (the kernels one
    # after the other, so that no launch shares the GPU with another), same L2 flushes
    plan_s = M.marfa_plan_create(lines, levels, [w.vmr for w in wls], rqs, outs, autotune=True, serial=True,
                                 stream=stream)
    M.marfa_plan_execute(plan_s, stream)
    kms = np.zeros(12)
    ev_s = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(float(i))
        ev_s[i][0].record(stream)
        M.marfa_plan_execute(plan_s, stream)
        ev_s[i][1].record(stream)
        kms += M.marfa_plan_info(plan_s, kernel_ms=True)[2]
    torch.cuda.synchronize()
    serial_ms = float(sum(a.elapsed_time(b) for a, b in ev_s)) / args.steps
    M.marfa_plan_destroy(plan_s)
    units_rank = sum(w.n_levels * n for w, n in zip(wls, npts))
    evals_job = int(sum_over_ranks(evals_per_step, dist, dev))
    value = job_throughput(units_job, 1, args.steps, t_total)
    evals_s = job_throughput(evals_job, 1, args.steps, t_total)

    # end to end through the public calls with host buffers (pinned): line records in,
    # prepare (the batch preparation for several requests), absorption (the batch call
    # for several requests), k(nu) back, every step
    rec_h = [torch.from_numpy(w.lines.view(np.uint8)).pin_memory().numpy().view(w.lines.dtype) for w in wls]
    out_h = [torch.empty((w.n_levels, n), dtype=torch.float32).pin_memory().numpy() for w, n in zip(wls, npts)]

    def e2e_step():
        if len(wls) == 1:
            l2 = [M.marfa_prepare_lines(rec_h[0], wls[0].species)]
            M.marfa_absorption(l2[0], levels[0], wls[0].vmr, rqs[0], out_h[0], stream)
        else:
            l2 = M.marfa_prepare_lines_batch(rec_h, [w.species for w in wls])
            M.marfa_absorption_batch(l2, levels, [w.vmr for w in wls], rqs, out_h, stream)
        for x in l2:
            M.marfa_free_lines(x)

    t_e2e = float("nan")
    if not args.no_e2e:
        e2e_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        t_e2e = max_over_ranks(time.perf_counter() - t0, dist, dev)
    e2e_value = job_throughput(units_job, 1, args.steps, t_e2e)

    # roofline of the dominant kernel (FP32 pipe, algorithmic flops per evaluation)
    names = ["level_prep"] + [f"grid{g}" for g in range(1, 11)] + ["finest"]
    dom = int(np.argmax(kms))
    dom_ms = kms[dom] / max(1, klaunch[dom])
    dom_flops = float(flops_grid[dom - 1]) if dom > 0 else 0.0
    evals_dom = float(counts_grid[dom - 1]) if dom > 0 else 0.0
    achieved = dom_flops / (dom_ms * 1e-3) / 1e12
    mhz, src = peaks()
    peak = N_SM * FP32_LANES * 2 * mhz * 1e6 / 1e12
    # measured issue rates beside the derived peak: FP32 FMA and the MUFU kinds the
    # Voigt branches use (ex2 in exp, rcp in the divisions, cos in the Gaussian core)
    probes = {"fp32_fma_tflops": 2.0 * M.marfa_diag_pipe_rate("fma") / 1e12}
    for k in ("ex2", "rcp", "cos"):
        probes[f"mufu_{k}_gops"] = M.marfa_diag_pipe_rate(k) / 1e9

    surr = None
    wpath = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2411_03418_gb300",
                         "surrogate_weights.npy")
    if args.workload == "venus" and not args.no_surrogate and os.path.exists(wpath):
        surr = surrogate_leg(args, M, wl, lines[0], levels[0], outs[0], flush, stream, wpath, evals_per_step,
                             ms_per_step, npts[0], dist, dev)

    if rank == 0:
        cfg = {"workload": wname, "requests": len(wls), "lines": int(sum(len(w.lines) for w in wls)),
               "levels": int(sum(w.n_levels for w in wls)), "points_x_levels_per_step": int(units_job),
               "l2": "flushed between steps (256 MB write)", "stencil": args.stencil}
        if len(wls) == 1:
            cfg["npts_per_level"] = npts[0]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak" if (world == 1 or shard == "none") else "strong", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": cfg,
            "line_evals_per_s": evals_s, "line_evals_per_step": evals_per_step,
            "line_evals_per_grid": [int(v) for v in counts_grid],
            "line_evals_class_per_grid": {"poly_cell": [int(v) for v in n_near],
                                          "asymptotic": [int(v) for v in n_mid],
                                          "small_y_cell": [int(v) for v in n_small]},
            "step_fp32_tflops": float(flops_grid.sum()) * world * args.steps / t_total / 1e12,
            "fp32_tflops_per_kernel": {n: (float(flops_grid[i - 1]) / (kms[i] / args.steps * 1e-3) / 1e12
                                           if i > 0 and kms[i] > 0 else None) for i, n in enumerate(names)},
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(sum(w.lines.nbytes + lv.nbytes + w.vmr.nbytes
                                                  for w, lv in zip(wls, levels))),
                    "d2h_bytes_per_step": int(sum(o.nbytes for o in out_h))},
            "gpu_launches": int(klaunch.sum()),
            "plan": {"graph": "one CUDA graph per step (12 kernel launches; grids 1-10 as parallel branches)",
                     "create_s": plan_s_create, "serial_ms_per_step": serial_ms,
                     "variant_grids_1_10_finest": [int(v) for v in variant],
                     "autotune_ms_per_launch": [[round(float(a), 3) for a in row] for row in tune_ms],
                     "size_classes": {"requests_per_class": [int((req_class == c).sum()) for c in range(2)],
                                      "choice_per_class": [[int(x) for x in row] for row in class_choice],
                                      "choice_layout": "[grid-1 split, variant of grids 2..10, finest variant]; "
                                                       "class 0: windows <= 16 cm-1, 1: wider; -1: no request"},
                     "variants": "grids 2-10: 0 line-major 32 pairs, 1 two-phase, 2 line-major 16 pairs, "
                                 "3 flattened, 4 by mechanism, 5 by mechanism merged; finest: 0 groups per panel, "
                                 "1 flattened jobs, 2 flattened jobs by mechanism, 3 the same with a merged edge/breakpoint pass"},
            "kernel_ms_per_step_serial": {n: float(kms[i] / args.steps) for i, n in enumerate(names)},
            "roofline": {"bound": "alu", "kernel": names[dom], "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": (TRAFFIC_BYTES.get((args.workload, names[dom], int(variant[dom - 1]) if dom > 0 else -1))
                                     if args.nu_lo is None and args.nu_hi is None and args.stencil == 3
                                     else None),
                         "flops_per_eval": {"far": FLOPS_FAR, "asymptotic": FLOPS_MID, "poly_cell": FLOPS_NEAR,
                                            "small_y_cell": FLOPS_SMALL},
                         "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz ({src} max clock)",
                         "frac_of_fma_probe": achieved / probes["fp32_fma_tflops"],
                         # the same launch with a flat 10 or 40 FP32 flops per evaluation (the
                         # per-evaluation range of the hot-path budget) instead of the
                         # implementation's counts by Voigt branch
                         "flat_10_40_flops_per_eval": {
                             "achieved": [evals_dom * f / (dom_ms * 1e-3) / 1e12 for f in (10.0, 40.0)],
                             "frac": [evals_dom * f / (dom_ms * 1e-3) / 1e12 / peak for f in (10.0, 40.0)]},
                         "probes": probes},
            "clocks": clocks,
        }
        if surr is not None:
            line["surrogate"] = surr
        if not args.no_cpu_baseline and world == 1 and args.workload == "venus":
            line["cpu_baseline"] = cpu_baseline_sample(wl)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
