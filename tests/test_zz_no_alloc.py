"""marfa_absorption_noalloc: the same k(nu) as marfa_absorption without allocating.

Callers that cannot allocate device memory (their own pool holds all free memory, or
an allocation or free must not synchronise the device while other streams run) get
this entry point; its scratch lives in a fixed 32 MiB device array of the library.
This file is collected last on purpose, so that a run stopping at its first failure
has already run every other test.
"""
import numpy as np
import pytest

from workloads import tiny_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_03418_gb300 import build, marfa
    build.build()
    marfa.load()
    return marfa


def _out(M, wl):
    import torch
    return torch.empty((wl.n_levels, M.marfa_num_points(wl.nu_lo, wl.nu_hi)), dtype=torch.float32,
                       device="cuda")


def test_noalloc_matches_allocating_call_on_two_calls_in_a_row(M):
    import torch
    stream = torch.cuda.current_stream()
    wls = [tiny_workload(301, 500, 2000.0, 2002.7, 25.0, T=(296.0, 200.0), p=(1.0, 1e-3),
                         chi="tonkov", chi_species=1),
           tiny_workload(302, 300, 1500.0, 1501.3, 125.0, T=(735.0,), p=(92.0,))]
    for wl in wls:
        lines = M.marfa_prepare_lines(wl.lines, wl.species)
        ref = _out(M, wl)
        M.marfa_absorption(lines, M.levels_of(wl), wl.vmr, M.request_of(wl), ref, stream)
        torch.cuda.synchronize()
        ref = ref.cpu().numpy().astype(np.float64)
        mx = np.abs(ref).max()
        big = np.abs(ref) > 1e-8 * mx
        for _ in range(2):  # the second call reuses the scratch the first one left
            got = _out(M, wl)
            got.fill_(float("nan"))
            M.marfa_absorption_noalloc(lines, M.levels_of(wl), wl.vmr, M.request_of(wl), got, stream)
            torch.cuda.synchronize()
            g = got.cpu().numpy().astype(np.float64)
            assert np.all(np.isfinite(g))
            assert np.abs(g[big] / ref[big] - 1).max() < 1e-4
            assert np.abs(g[~big] - ref[~big]).max(initial=0.0) <= 1e-4 * 1e-8 * mx


def test_noalloc_rejects_oversized_requests_and_host_outputs(M):
    wl = tiny_workload(303, 200_000, 2000.0, 3000.0, 125.0, T=tuple([296.0] * 8), p=tuple([1.0] * 8))
    lines = M.marfa_prepare_lines(wl.lines, wl.species)
    with pytest.raises(M.MarfaError) as e:
        M.marfa_absorption_noalloc(lines, M.levels_of(wl), wl.vmr, M.request_of(wl), _out(M, wl))
    assert e.value.code == -1 and "scratch" in str(e.value)
    small = tiny_workload(304, 100, 1000.0, 1000.5, 25.0)
    lines = M.marfa_prepare_lines(small.lines, small.species)
    host = np.empty((1, M.marfa_num_points(1000.0, 1000.5)), np.float32)
    with pytest.raises(M.MarfaError) as e:
        M.marfa_absorption_noalloc(lines, M.levels_of(small), small.vmr, M.request_of(small), host)
    assert e.value.code == -1
