"""Dense parity at full size: the Venus workload (200,000 lines, 60 levels, Voigt x
Tonkov chi, 125 cm^-1 cut-off, 2000-3000 cm^-1) through the captured, autotuned plan
the benchmark times, plain and with the learned surrogate, against the FP64 oracle's
eleven-grid sum on contiguous 1 cm^-1 sub-windows (2,049 nodes each) at five levels.

The sub-windows: one straddling a grid-1 tile edge (tiles of 32 pairs = 64 cm^-1 start at
2000 + 64 k), one starting 3 cm^-1 above the strongest line (every line of that band
puts a chi breakpoint near it), one at the window centre and the last one of the window.
The oracle runs on the lines within reach of each sub-window, one spawned process per
(level, sub-window). Bars: 1e-4 relative for the plain path and 1e-3 for the surrogate
path wherever k exceeds 1e-8 of the level's maximum (absolute floor below); the max and
RMS relative errors of every (level, sub-window) are printed.
"""
import os
from concurrent.futures import ProcessPoolExecutor
import multiprocessing as mp

import numpy as np
import pytest

from oracle import marfa_oracle as O
from workloads import config1_venus

pytestmark = pytest.mark.gpu

FLOOR = 1e-8
LEVELS = (0, 15, 30, 45, 59)
WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_2411_03418_gb300", "surrogate_weights.npy")


def _sub_oracle(args):
    """The oracle's eleven-grid sum on one sub-window of one level (spawned worker)."""
    lev, lo, hi = args
    wl = config1_venus()
    sel = np.abs(wl.lines["nu0"] - 0.5 * (lo + hi)) <= 0.5 * (hi - lo) + wl.cutoff + 2.0
    sub = wl.with_(lines=wl.lines[sel], nu_lo=lo, nu_hi=hi).level_subset([lev])
    return O.eleven_grid(sub, 0)


@pytest.fixture(scope="module")
def M():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_03418_gb300 import build, marfa
    build.build()
    marfa.load()
    return marfa


@pytest.fixture(scope="module")
def venus():
    wl = config1_venus()
    strongest = float(wl.lines["nu0"][np.argmax(wl.lines["S296"] * ((wl.lines["nu0"] > 2010) & (wl.lines["nu0"] < 2985)))])
    starts = [2063.5, np.floor((strongest + 3.0) * 2048) / 2048, 2500.0, 2999.0]
    jobs = [(lev, lo, lo + 1.0) for lev in LEVELS for lo in starts]
    with ProcessPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 1),
                             mp_context=mp.get_context("spawn")) as ex:
        refs = list(ex.map(_sub_oracle, jobs))
    return wl, jobs, refs


def _run_plan(M, wl):
    import torch
    lines = M.marfa_prepare_lines(wl.lines, wl.species)
    n = M.marfa_num_points(wl.nu_lo, wl.nu_hi)
    out = torch.full((wl.n_levels, n), float("nan"), dtype=torch.float32, device="cuda")
    plan = M.marfa_plan_create([lines], [M.levels_of(wl)], [wl.vmr], [M.request_of(wl)], [out], autotune=True)
    out.fill_(float("nan"))
    M.marfa_plan_execute(plan)
    torch.cuda.synchronize()
    M.marfa_plan_destroy(plan)
    assert not torch.isnan(out).any()
    return out


def _compare(out, wl, jobs, refs, rtol, what):
    k_lo, _ = O.window_nodes(wl.nu_lo, wl.nu_hi)
    # the floor from the oracle alone: its largest value over the level's sub-windows (a
    # lower bound of the level's maximum: the floor can only be stricter than defined)
    rowmax = {lev: max(float(np.abs(r).max()) for (l, _, _), r in zip(jobs, refs) if l == lev) for lev in LEVELS}
    report, worst = [], 0.0
    for (lev, lo, hi), ref in zip(jobs, refs):
        i0 = int(round(lo * 2048)) - k_lo
        got = out[lev, i0:i0 + len(ref)].cpu().numpy().astype(np.float64)
        assert len(got) == len(ref) == 2049
        big = np.abs(ref) > FLOOR * rowmax[lev]
        rel = np.abs(got[big] / ref[big] - 1.0)
        report.append((lev, lo, rel.max(), float(np.sqrt(np.mean(rel ** 2))), int(big.sum())))
        worst = max(worst, rel.max())
        assert rel.max() < rtol, f"{what}: level {lev} window {lo}: max rel err {rel.max():.3e}"
        if (~big).any():
            assert np.abs(got[~big] - ref[~big]).max() <= rtol * FLOOR * rowmax[lev], f"{what}: floor"
    print(f"\n{what} vs the FP64 oracle (level, sub-window start, max rel, rms rel, nodes above floor):")
    for r in report:
        print(f"  {r[0]:2d} {r[1]:9.4f} {r[2]:.3e} {r[3]:.3e} {r[4]}")
    return worst


def test_venus_plan_dense_subwindows(M, venus):
    wl, jobs, refs = venus
    out = _run_plan(M, wl)
    _compare(out, wl, jobs, refs, 1e-4, "Venus plan (plain)")


def test_venus_surrogate_plan_dense_subwindows(M, venus):
    if not os.path.exists(WEIGHTS):
        pytest.skip("trained surrogate parameters not present")
    wl, jobs, refs = venus
    M.marfa_surrogate_load(np.load(WEIGHTS).astype(np.float32), 6e-4, 32)
    try:
        out = _run_plan(M, wl.with_(surrogate=1))
    finally:
        M.marfa_surrogate_unload()
    _compare(out, wl, jobs, refs, 1e-3, "Venus plan (surrogate)")
