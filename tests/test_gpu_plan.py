"""Captured plans (one CUDA graph per batch, optional per-grid kernel autotuning) and the
full-size batch and Earth workloads, against the FP64 oracle on the GPU.

Bars as in test_gpu_parity: 1e-4 relative on k(nu) wherever k exceeds 1e-8 of the row
maximum, an absolute floor below; bit-identical where the same kernels run in the same
order (plan without tuning vs marfa_absorption_batch, replays of one plan)."""
import numpy as np
import pytest

from oracle import marfa_oracle as O
from workloads import config1_venus, config2_batch, config3_earth, tiny_workload

pytestmark = pytest.mark.gpu

RTOL = 1e-4
FLOOR = 1e-8


@pytest.fixture(scope="module")
def M():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_03418_gb300 import build, marfa
    build.build()
    marfa.load()
    return marfa


def peak_node(wl, lev, k_lo):
    """Index (from k_lo) of the finest node nearest the centre of the line with the highest
    peak inside the window at level lev (from the oracle's level parameters), or 0: with it
    in a sample, the sample's largest oracle value bounds the level's maximum from below,
    so a floor taken from it can only be stricter than the definition's."""
    P = O.level_params(wl, lev)
    inside = (P["nu_shift"] > wl.nu_lo) & (P["nu_shift"] < wl.nu_hi)
    if not inside.any():
        return 0
    peak = np.where(inside, P["amp"] / np.maximum(P["alpha_D"], P["gamma_L"]), 0.0)
    return int(np.rint(P["nu_shift"][int(np.argmax(peak))] * 2048)) - k_lo


def check(got, ref, rowmax, what):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    big = np.abs(ref) > FLOOR * rowmax
    if big.any():
        rel = np.abs(got[big] / ref[big] - 1)
        assert rel.max() < RTOL, f"{what}: max rel err {rel.max():.3e}"
    if (~big).any():
        assert np.abs(got[~big] - ref[~big]).max() <= RTOL * FLOOR * rowmax, f"{what}: floor"


SMALL = [
    tiny_workload(41, 300, 2000.0, 2003.0, 25.0, T=(735.0, 296.0, 170.0), p=(92.0, 1.0, 1e-5),
                  chi="tonkov", chi_species=1),
    tiny_workload(42, 120, 4000.0, 4000.25, 10.0, T=(250.0,), p=(0.05,), spread=3.0),
    tiny_workload(43, 500, 1000.0, 1010.0, 125.0, T=(400.0, 200.0), p=(5.0, 1e-3), shape="lorentz"),
]


def _batch_and_plan(M, wls, autotune):
    import torch
    lines = [M.marfa_prepare_lines(w.lines, w.species) for w in wls]
    lv = [M.levels_of(w) for w in wls]
    rq = [M.request_of(w) for w in wls]
    ref = [np.empty((w.n_levels, M.marfa_num_points(w.nu_lo, w.nu_hi)), np.float32) for w in wls]
    M.marfa_absorption_batch(lines, lv, [w.vmr for w in wls], rq, ref)
    outs = [torch.full(r.shape, float("nan"), dtype=torch.float32, device="cuda") for r in ref]
    plan = M.marfa_plan_create(lines, lv, [w.vmr for w in wls], rq, outs, autotune=autotune)
    return plan, ref, outs


def test_plan_matches_batch_and_replays(M):
    import torch
    plan, ref, outs = _batch_and_plan(M, SMALL, autotune=False)
    for r, o in zip(ref, outs):  # creation leaves the result in place
        assert np.array_equal(o.cpu().numpy(), r)
    for o in outs:
        o.fill_(float("nan"))
    s = torch.cuda.Stream()
    for _ in range(2):
        M.marfa_plan_execute(plan, s)
    s.synchronize()
    for r, o in zip(ref, outs):
        assert np.array_equal(o.cpu().numpy(), r)
    v, t, k = M.marfa_plan_info(plan, kernel_ms=True)
    assert list(v) == list(M.marfa_diag_variants())  # the process-wide defaults
    assert np.all(t == -1)
    assert np.all(k >= 0) and k.sum() > 0
    M.marfa_plan_destroy(plan)


def test_five_point_plan_matches_batch(M):
    """The 5-point variant through a captured plan equals marfa_absorption_batch."""
    import torch
    wls = [w.with_(stencil=5) for w in SMALL]
    plan, ref, outs = _batch_and_plan(M, wls, autotune=False)
    M.marfa_plan_execute(plan)
    torch.cuda.synchronize()
    for r, o in zip(ref, outs):
        assert np.array_equal(o.cpu().numpy(), r)
    M.marfa_plan_destroy(plan)


def test_mixed_stencils_rejected(M):
    """The plain kernels are compiled for one partition: a call mixing 3- and 5-point
    requests is refused."""
    import torch
    wls = [SMALL[0], SMALL[1].with_(stencil=5)]
    lines = [M.marfa_prepare_lines(w.lines, w.species) for w in wls]
    outs = [torch.empty((w.n_levels, M.marfa_num_points(w.nu_lo, w.nu_hi)), dtype=torch.float32, device="cuda")
            for w in wls]
    with pytest.raises(M.MarfaError, match="stencil"):
        M.marfa_absorption_batch(lines, [M.levels_of(w) for w in wls], [w.vmr for w in wls],
                                 [M.request_of(w) for w in wls], outs)


def test_autotuned_plan_parity(M):
    import torch
    plan, ref, outs = _batch_and_plan(M, SMALL, autotune=True)
    M.marfa_plan_execute(plan)
    torch.cuda.synchronize()
    v, t, _ = M.marfa_plan_info(plan)
    assert set(v[1:10].tolist()) <= {0, 1, 2, 3, 4, 5} and v[10] in (0, 1, 2, 3)
    assert np.all(t[1:10] > 0) and np.all(t[10, :4] > 0) and np.all(t[10, 4:] == -1) and np.all(t[0] == -1)
    for g in range(1, 10):  # the chosen variant is the fastest one
        assert t[g, v[g]] <= t[g].min()
    assert t[10, v[10]] <= t[10, :4].min()
    for q, w in enumerate(SMALL):
        got = outs[q].cpu().numpy()
        for lev in range(w.n_levels):
            check(got[lev], O.eleven_grid(w, lev), np.abs(got[lev]).max(), f"request {q} level {lev}")
            # another summation order of the same terms: within FP32 rounding of the batch result
            check(got[lev], ref[q][lev], np.abs(got[lev]).max(), f"request {q} level {lev} vs batch")


def test_pinned_host_output_matches_device_output(M):
    """A page-locked host k_out is written by the kernels directly; pageable host memory
    goes through a device buffer and a copy. All three give the same bytes."""
    import torch
    w = SMALL[0]
    lines = M.marfa_prepare_lines(w.lines, w.species)
    shape = (w.n_levels, M.marfa_num_points(w.nu_lo, w.nu_hi))
    dev = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
    M.marfa_absorption(lines, M.levels_of(w), w.vmr, M.request_of(w), dev)
    torch.cuda.synchronize()
    pinned = torch.full(shape, float("nan"), dtype=torch.float32).pin_memory().numpy()
    pageable = np.full(shape, np.nan, dtype=np.float32)
    for _ in range(2):  # twice: the second call overwrites the first call's result
        M.marfa_absorption(lines, M.levels_of(w), w.vmr, M.request_of(w), pinned)
        M.marfa_absorption(lines, M.levels_of(w), w.vmr, M.request_of(w), pageable)
        ref = dev.cpu().numpy()
        assert np.array_equal(pinned, ref)
        assert np.array_equal(pageable, ref)
        pinned[:] = np.nan
        pageable[:] = np.nan


def test_plan_rejects_host_outputs(M):
    w = SMALL[1]
    lines = [M.marfa_prepare_lines(w.lines, w.species)]
    out = np.empty((w.n_levels, M.marfa_num_points(w.nu_lo, w.nu_hi)), np.float32)
    with pytest.raises(M.MarfaError, match="device memory"):
        M.marfa_plan_create(lines, [M.levels_of(w)], [w.vmr], [M.request_of(w)], [out])


# ------------------------------------------------------------ full-size workloads, sampled
def test_config1_venus_autotuned_plan_sampled(M):
    """The launch configuration bench.py times: the Venus workload as one autotuned plan."""
    import torch
    wl = config1_venus()
    lines = M.marfa_prepare_lines(wl.lines, wl.species)
    n = M.marfa_num_points(wl.nu_lo, wl.nu_hi)
    out = torch.empty((wl.n_levels, n), dtype=torch.float32, device="cuda")
    plan = M.marfa_plan_create([lines], [M.levels_of(wl)], [wl.vmr], [M.request_of(wl)], [out], autotune=True)
    out.fill_(float("nan"))
    M.marfa_plan_execute(plan)
    torch.cuda.synchronize()
    rng = np.random.default_rng(6)
    k_lo, _ = O.window_nodes(wl.nu_lo, wl.nu_hi)
    for lev in (0, 29, 59):
        idx = np.concatenate([[0, n - 1, peak_node(wl, lev, k_lo)], rng.integers(0, n, 10)])
        ref = O.eleven_grid_at(wl, lev, k_lo + idx)
        got = out[lev, torch.as_tensor(idx, device="cuda")].cpu().numpy()
        check(got, ref, float(np.abs(ref).max()), f"Venus level {lev}")
    assert not torch.isnan(out).any()
    M.marfa_plan_destroy(plan)


def test_config2_batch_full_size(M):
    """256 uneven requests in one autotuned plan (one graph); sampled nodes of every
    other request against the oracle, and the plan against marfa_absorption_batch."""
    import torch
    wls = config2_batch()
    assert len(wls) == 256
    lines = [M.marfa_prepare_lines(w.lines, w.species) for w in wls]
    lv = [M.levels_of(w) for w in wls]
    rq = [M.request_of(w) for w in wls]
    outs = [torch.empty((w.n_levels, M.marfa_num_points(w.nu_lo, w.nu_hi)), dtype=torch.float32, device="cuda")
            for w in wls]
    plan = M.marfa_plan_create(lines, lv, [w.vmr for w in wls], rq, outs, autotune=True)
    for o in outs:
        o.fill_(float("nan"))
    M.marfa_plan_execute(plan)
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    for q in range(0, 256, 8):
        w = wls[q]
        n = outs[q].shape[1]
        k_lo, _ = O.window_nodes(w.nu_lo, w.nu_hi)
        lev = int(rng.integers(0, w.n_levels))
        idx = np.array([0, n - 1, int(rng.integers(0, n)), peak_node(w, lev, k_lo)])
        ref = O.eleven_grid_at(w, lev, k_lo + idx)
        got = outs[q][lev, torch.as_tensor(idx, device="cuda")].cpu().numpy()
        check(got, ref, float(np.abs(ref).max()), f"request {q} level {lev}")
    # the whole batch through marfa_absorption_batch (default kernels), device outputs
    ref = [torch.empty_like(o) for o in outs]
    M.marfa_absorption_batch(lines, lv, [w.vmr for w in wls], rq, ref, torch.cuda.current_stream())
    torch.cuda.synchronize()
    for q in range(256):
        r, o = ref[q], outs[q]
        assert not torch.isnan(o).any()
        mx = r.abs().amax(dim=1, keepdim=True)
        big = r.abs() > FLOOR * mx
        rel = ((o - r).abs() / r.abs().clamp_min(1e-38))[big]
        assert rel.numel() == 0 or float(rel.max()) < 1e-5, f"request {q}"
    M.marfa_plan_destroy(plan)


def test_config3_earth_precision(M):
    """Earth-like mixture (1.2M lines, 50 levels, 500-3000 cm^-1): the FP32 compensated
    path against the FP64 eleven-grid oracle on 0.5 cm^-1 sub-windows of ten levels, with
    the max and RMS relative error per level printed."""
    import torch
    wl = config3_earth()
    lines = M.marfa_prepare_lines(wl.lines, wl.species)
    n = M.marfa_num_points(wl.nu_lo, wl.nu_hi)
    out = torch.empty((wl.n_levels, n), dtype=torch.float32, device="cuda")
    plan = M.marfa_plan_create([lines], [M.levels_of(wl)], [wl.vmr], [M.request_of(wl)], [out], autotune=True)
    M.marfa_plan_execute(plan)
    torch.cuda.synchronize()
    assert not torch.isnan(out).any()
    k_lo, _ = O.window_nodes(wl.nu_lo, wl.nu_hi)
    rng = np.random.default_rng(8)
    report = []
    for lev in range(0, wl.n_levels, 5):
        lo = float(np.round(rng.uniform(510.0, 2990.0) * 4) / 4)
        sel = (wl.lines["nu0"] > lo - wl.cutoff - 2.0) & (wl.lines["nu0"] < lo + 0.5 + wl.cutoff + 2.0)
        sub = wl.with_(lines=wl.lines[sel], nu_lo=lo, nu_hi=lo + 0.5).level_subset([lev])
        ref = O.eleven_grid(sub, 0)
        i0 = int(round(lo * 2048)) - k_lo
        got = out[lev, i0:i0 + len(ref)].cpu().numpy().astype(np.float64)
        rowmax = float(np.abs(ref).max())  # the oracle's: a lower bound, so a stricter floor
        check(got, ref, rowmax, f"Earth level {lev} at {lo}")
        big = np.abs(ref) > FLOOR * rowmax
        rel = np.abs(got[big] / ref[big] - 1)
        report.append((lev, lo, rel.max(), np.sqrt(np.mean(rel ** 2))))
    print("\nEarth precision (level, window start, max rel, rms rel):")
    for r in report:
        print(f"  {r[0]:2d} {r[1]:8.2f} {r[2]:.3e} {r[3]:.3e}")
    M.marfa_plan_destroy(plan)


def test_pipe_rate_probes(M):
    """The issue-rate probes behind the roofline: FP32 FMA near 128 a clock per SM, the
    MUFU kinds well below it."""
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    fma = M.marfa_diag_pipe_rate("fma")
    assert 0.3e9 * nsm * 128 < fma < 2.2e9 * nsm * 128 * 1.05
    for k in ("ex2", "rcp", "cos"):
        r = M.marfa_diag_pipe_rate(k)
        assert 0.0 < r < fma / 2


def test_size_classes_tuned_apart(M):
    """A batch of narrow (<= 16 cm^-1) and wide windows: each request gets its size class,
    each class its own grid-1 split and kernel variants (the fastest of the autotuner's
    timings on that class's work), and the plan stays within FP32 rounding of the
    untuned batch and within 1e-4 of the oracle."""
    import torch
    wls = [tiny_workload(44, 300, 2000.0, 2003.0, 25.0, T=(400.0, 200.0), p=(5.0, 1e-3), chi="tonkov",
                         chi_species=1),
           tiny_workload(45, 400, 3000.0, 3020.5, 25.0, T=(296.0,), p=(0.1,)),
           tiny_workload(46, 200, 1200.0, 1201.0, 10.0, T=(250.0,), p=(0.05,))]
    plan, ref, outs = _batch_and_plan(M, wls, autotune=True)
    M.marfa_plan_execute(plan)
    torch.cuda.synchronize()
    rc, ch, t = M.marfa_plan_classes(plan, len(wls))
    assert list(rc) == [0, 1, 0]
    splits = [1, 2, 3, 6]
    for c in (0, 1):
        assert ch[c, 0] in splits
        assert ch[c, 0] == splits[int(np.argmin(t[c, 0, :4]))]
        assert np.all(t[c, 0, :4] > 0) and np.all(t[c, 0, 4:] == -1)
        for g in range(1, 10):
            assert 0 <= ch[c, g] <= 5 and t[c, g, ch[c, g]] <= t[c, g].min()
        assert 0 <= ch[c, 10] <= 3 and t[c, 10, ch[c, 10]] <= t[c, 10, :4].min()
    v, _, _ = M.marfa_plan_info(plan)
    assert list(v[1:]) == list(ch[rc[0], 1:])  # plan_info reports request 0's class
    for q, w in enumerate(wls):
        got = outs[q].cpu().numpy()
        for lev in range(w.n_levels):
            check(got[lev], ref[q][lev], np.abs(got[lev]).max(), f"request {q} level {lev} vs batch")
            check(got[lev], O.eleven_grid(w, lev), np.abs(got[lev]).max(), f"request {q} level {lev}")
    M.marfa_plan_destroy(plan)


def test_batch_preparation_equals_single_preparation(M):
    """marfa_prepare_lines_batch gives every request the list marfa_prepare_lines makes:
    the batch computed from either set of handles is the same bit for bit. A request with
    an invalid record fails the whole call, naming that request, with nothing held."""
    wls = [tiny_workload(300 + q, 150 + 40 * q, 1500.0 + 3 * q, 1501.2 + 3 * q, 25.0, T=(296.0, 200.0),
                         p=(1.0, 1e-3), chi="tonkov", chi_species=1) for q in range(5)]
    single = [M.marfa_prepare_lines(w.lines, w.species) for w in wls]
    batch = M.marfa_prepare_lines_batch([w.lines for w in wls], [w.species for w in wls])
    outs = []
    for handles in (single, batch):
        o = [np.empty((w.n_levels, M.marfa_num_points(w.nu_lo, w.nu_hi)), np.float32) for w in wls]
        M.marfa_absorption_batch(handles, [M.levels_of(w) for w in wls], [w.vmr for w in wls],
                                 [M.request_of(w) for w in wls], o)
        outs.append(o)
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    used0 = M.marfa_diag_device_memory()[0]
    bad = wls[3].lines.copy()
    bad["nu0"][7] = np.nan
    with pytest.raises(M.MarfaError, match="request 3"):
        M.marfa_prepare_lines_batch([w.lines for w in wls[:3]] + [bad, wls[4].lines], [w.species for w in wls])
    assert M.marfa_diag_device_memory()[0] == used0
