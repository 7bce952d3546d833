"""marfa_absorption_noalloc: the same k(nu) as marfa_absorption without allocating.

Callers that cannot allocate device memory (their own pool holds all free memory, or
an allocation or free must not synchronise the device while other streams run) get
this entry point; its scratch lives in a fixed 32 MiB device array of the library,
which a device commits when marfa_prepare_lines first runs there.
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


def _compare_two_calls(M, wl):
    """marfa_absorption's k(nu), then marfa_absorption_noalloc twice in a row on the same
    request: both calls within 1e-4 of it (absolute floor below 1e-8 of the maximum)."""
    import torch
    stream = torch.cuda.current_stream()
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


def test_noalloc_matches_allocating_call_on_two_calls_in_a_row(M):
    _compare_two_calls(M, tiny_workload(301, 500, 2000.0, 2002.7, 25.0, T=(296.0, 200.0), p=(1.0, 1e-3),
                                        chi="tonkov", chi_species=1))
    _compare_two_calls(M, tiny_workload(302, 300, 1500.0, 1501.3, 125.0, T=(735.0,), p=(92.0,)))


def test_noalloc_five_point_stencil(M):
    """The 5-point variant takes its own kernel instantiations and slot ranges."""
    _compare_two_calls(M, tiny_workload(305, 400, 2000.0, 2001.9, 25.0, T=(296.0, 200.0), p=(1.0, 1e-3),
                                        chi="tonkov", chi_species=1, stencil=5))


def test_noalloc_with_the_surrogate(M):
    """A surrogate request takes the surrogate-capable kernels (network weights and
    queues in shared memory)."""
    import os
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "paper_2411_03418_gb300", "surrogate_weights.npy")
    if not os.path.exists(path):
        pytest.skip("trained surrogate parameters not present")
    M.marfa_surrogate_load(np.load(path).astype(np.float32), 6e-4, 32)
    try:
        _compare_two_calls(M, tiny_workload(306, 400, 2400.0, 2401.5, 25.0, T=(400.0, 170.0),
                                            p=(1e-2, 1e-5), chi="tonkov", chi_species=1).with_(surrogate=1))
    finally:
        M.marfa_surrogate_unload()


def test_noalloc_refuses_a_stream_in_capture(M):
    """The call copies its tables from host memory it frees on return, so a stream in
    capture is refused before any work is queued."""
    import torch
    wl = tiny_workload(307, 100, 1000.0, 1000.5, 25.0)
    lines = M.marfa_prepare_lines(wl.lines, wl.species)
    out = _out(M, wl)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(M.MarfaError) as e:
        with torch.cuda.graph(g, stream=s):
            M.marfa_absorption_noalloc(lines, M.levels_of(wl), wl.vmr, M.request_of(wl), out, s)
    assert e.value.code == -1 and "capture" in str(e.value)
    torch.cuda.synchronize()


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
