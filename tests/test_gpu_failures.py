"""Error paths of the entry points on the GPU: with the allocation-failure injector armed
at the n-th allocation (n = 1, 2, ... until the call goes through), every entry point
returns MARFA_E_NOMEM, frees what it had allocated (the device pool's bytes in use and
the free device memory come back to where they were) and leaves the library usable (the
same call then gives the reference result bit for bit)."""
import os

import numpy as np
import pytest

from workloads import tiny_workload

pytestmark = pytest.mark.gpu

NOMEM = -2
WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_2411_03418_gb300", "surrogate_weights.npy")


@pytest.fixture(scope="module")
def M():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_03418_gb300 import build, marfa
    build.build()
    marfa.load()
    yield marfa
    marfa.marfa_diag_fail_alloc(0)


WL = tiny_workload(201, 300, 2000.0, 2001.5, 25.0, T=(296.0, 200.0), p=(1.0, 1e-3), chi="tonkov", chi_species=1)
WL2 = tiny_workload(202, 200, 1500.0, 1500.7, 10.0, T=(250.0,), p=(0.1,))


def _exhaust(M, call, what, device_free=False):
    """Arm the injector at n = 1, 2, ... until `call` succeeds; returns (allocations
    the call makes, its result). Every failing run must raise MARFA_E_NOMEM and leave
    the device pool's bytes in use as they were (and, with device_free, the free device
    memory too: for calls whose failing runs must not reserve device memory at all; the
    pool keeps what it has reserved, so the free memory is no leak measure once a call
    has taken pool memory)."""
    import gc
    gc.collect()
    used, free = M.marfa_diag_device_memory()
    base = (used, free) if device_free else (used,)
    for n in range(1, 200):
        M.marfa_diag_fail_alloc(n)
        try:
            res = call()
        except M.MarfaError as e:
            assert e.code == NOMEM, f"{what}: allocation {n}: {e}"
            assert M.marfa_diag_fail_alloc(0) == 0  # the injector fired and disarmed
            gc.collect()
            now = M.marfa_diag_device_memory()
            assert now[:len(base)] == base, f"{what}: allocation {n} leaked"
            continue
        assert M.marfa_diag_fail_alloc(0) > 0  # this run made fewer than n allocations
        return n - 1, res
    raise AssertionError(f"{what} never completed")


def _direct(M, lines, wl, out):
    import torch
    M.marfa_absorption(lines, M.levels_of(wl), wl.vmr, M.request_of(wl), out, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return out if isinstance(out, np.ndarray) else out.cpu().numpy()


def test_every_entry_point_fails_cleanly_and_recovers(M):
    import torch
    n = M.marfa_num_points(WL.nu_lo, WL.nu_hi)
    lines = M.marfa_prepare_lines(WL.lines, WL.species)
    dev = torch.empty((WL.n_levels, n), dtype=torch.float32, device="cuda")
    pageable = np.empty((WL.n_levels, n), np.float32)
    pinned = torch.empty((WL.n_levels, n), dtype=torch.float32).pin_memory().numpy()
    # warm up every kernel once (their modules load on first use, which takes memory)
    ref = _direct(M, lines, WL, dev).copy()
    _direct(M, lines, WL, pageable)
    _direct(M, lines, WL, pinned)
    plan = M.marfa_plan_create([lines], [M.levels_of(WL)], [WL.vmr], [M.request_of(WL)], [dev], autotune=True)
    M.marfa_plan_destroy(plan)
    del plan

    k, made = _exhaust(M, lambda: M.marfa_prepare_lines(WL.lines, WL.species), "marfa_prepare_lines",
                       device_free=True)
    assert k >= 3  # line-list object, host staging buffer, device block
    del made
    for out, name in ((dev, "device output"), (pageable, "pageable host output"), (pinned, "pinned host output")):
        k, got = _exhaust(M, lambda: _direct(M, lines, WL, out), f"marfa_absorption, {name}")
        assert k >= 2 and np.array_equal(got, ref), name
    def prep_batch():
        got = M.marfa_prepare_lines_batch([WL.lines, WL2.lines, WL.lines], [WL.species, WL2.species, WL.species])
        assert len(got) == 3
        return got
    k, made = _exhaust(M, prep_batch, "marfa_prepare_lines_batch")
    assert k >= 9  # three lists: object, host staging buffer, device block each
    del made
    lines2 = M.marfa_prepare_lines(WL2.lines, WL2.species)
    outs = [np.empty((w.n_levels, M.marfa_num_points(w.nu_lo, w.nu_hi)), np.float32) for w in (WL, WL2)]

    def batch():
        M.marfa_absorption_batch([lines, lines2], [M.levels_of(WL), M.levels_of(WL2)], [WL.vmr, WL2.vmr],
                                 [M.request_of(WL), M.request_of(WL2)], outs)
        return outs[0].copy()
    k, got = _exhaust(M, batch, "marfa_absorption_batch")
    assert k >= 3 and np.array_equal(got, ref)

    def make_plan():
        dev.fill_(float("nan"))
        p = M.marfa_plan_create([lines], [M.levels_of(WL)], [WL.vmr], [M.request_of(WL)], [dev])
        M.marfa_plan_execute(p)
        torch.cuda.synchronize()
        M.marfa_plan_destroy(p)
        return dev.cpu().numpy()
    k, got = _exhaust(M, make_plan, "marfa_plan_create")
    assert k >= 3 and np.array_equal(got, ref)

    def tuned_plan():
        p = M.marfa_plan_create([lines], [M.levels_of(WL)], [WL.vmr], [M.request_of(WL)], [dev], autotune=True)
        M.marfa_plan_destroy(p)
        return True
    k, _ = _exhaust(M, tuned_plan, "marfa_plan_create (autotune)")
    assert k >= 4

    if os.path.exists(WEIGHTS):
        w = np.load(WEIGHTS).astype(np.float32)
        k, _ = _exhaust(M, lambda: M.marfa_surrogate_load(w, 6e-4, 32), "marfa_surrogate_load")
        assert k >= 1
        M.marfa_surrogate_unload()
    # usable afterwards: the reference result again
    assert np.array_equal(_direct(M, lines, WL, dev), ref)
