"""The C-ABI library builds, loads without a GPU and exports what include/marfa.h
declares; host-only entry points (PT-table writer, argument validation) checked on CPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import marfa_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def M():
    from paper_2411_03418_gb300 import build, marfa
    build.build()
    marfa.load()
    return marfa


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "marfa.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(marfa_[a-z_]+)\s*\(", txt)))


def test_header_and_library_exports_agree(M):
    syms = declared_symbols()
    assert len(syms) >= 11
    lib = ctypes.CDLL(M.lib_path())
    for s in syms:
        assert hasattr(lib, s), f"{s} declared in include/marfa.h but not exported"
    assert sorted(M.EXPORTS) == syms


def test_struct_layouts(M):
    assert M.LINE_DTYPE.itemsize == 36
    assert M.SPECIES_DTYPE.itemsize == 24
    assert ctypes.sizeof(M.marfa_request_t) == 56


def test_num_points_matches_oracle(M):
    for lo, hi in [(4000, 4010), (2000, 3000), (999.13, 1001.0), (0.0, 0.0001), (5.0, 4.0),
                   (123.456, 123.457)]:
        assert M.marfa_num_points(lo, hi) == O.num_points(lo, hi)
    assert M.marfa_num_points(-1.0, 2.0) < 0
    assert M.marfa_num_points(float("nan"), 2.0) < 0


def test_pt_table_bytes_match_appendix_a_layout(M, tmp_path):
    rng = np.random.default_rng(0)
    n = O.num_points(20.0, 50.0)
    k = rng.random(n).astype(np.float32)
    M.marfa_write_pt_table(str(tmp_path), 7, 20.0, 50.0, k)
    data = (tmp_path / "7__.ptbin").read_bytes()
    assert data == O.pt_table_bytes(20.0, 50.0, k)
    M.marfa_write_pt_table(str(tmp_path), 123, 20.0, 50.0, k)
    assert (tmp_path / "123.ptbin").exists()


@pytest.mark.parametrize("args", [(19.0, 50.0), (20.0, 20.0), (25.0, 50.0)])
def test_pt_table_rejects_bad_windows(M, tmp_path, args):
    k = np.zeros(10, dtype=np.float32)
    with pytest.raises(M.MarfaError) as e:
        M.marfa_write_pt_table(str(tmp_path), 1, args[0], args[1], k)
    assert e.value.code == -1


def test_pt_table_io_error(M):
    n = O.num_points(20.0, 30.0)
    with pytest.raises(M.MarfaError) as e:
        M.marfa_write_pt_table("/nonexistent/dir/for/ptbin", 1, 20.0, 30.0, np.zeros(n, np.float32))
    assert e.value.code == -4


def test_prepare_lines_validation_before_any_device_call(M):
    from workloads import config0_tiny
    wl = config0_tiny()
    bad = wl.lines.copy()
    bad["nu0"][3] = np.nan
    with pytest.raises(M.MarfaError) as e:
        M.marfa_prepare_lines(bad, wl.species)
    assert e.value.code == -1 and "nu0" in str(e.value)
    bad = wl.lines.copy()
    bad["mol_iso"][5] = 99
    with pytest.raises(M.MarfaError):
        M.marfa_prepare_lines(bad, wl.species)
    sp2 = np.concatenate([wl.species, wl.species])
    with pytest.raises(M.MarfaError) as e:
        M.marfa_prepare_lines(wl.lines, sp2)
    assert "duplicate" in str(e.value)
    with pytest.raises(M.MarfaError):
        M.marfa_prepare_lines(wl.lines[:0], wl.species)


def test_prepare_lines_reports_first_invalid_line(M):
    """Validation runs over chunks of the line list on several host threads; the error
    names the first invalid line whatever chunk it falls in."""
    from workloads import config0_tiny
    wl = config0_tiny()
    big = np.resize(wl.lines, 200_003)
    bad = big.copy()
    bad["nu0"][150_001] = -1.0
    bad["mol_iso"][170_000] = 99
    bad["S296"][199_999] = np.inf
    for first, what in [(150_001, "nu0"), (170_000, "unknown species"), (199_999, "non-finite")]:
        with pytest.raises(M.MarfaError) as e:
            M.marfa_prepare_lines(bad, wl.species)
        assert e.value.code == -1 and f"line {first}:" in str(e.value) and what in str(e.value)
        bad["nu0"][150_001] = 1.0
        if first >= 170_000:
            bad["mol_iso"][170_000] = wl.lines["mol_iso"][0]
    bad2 = big.copy()
    bad2["gamma_air"][7] = np.nan
    bad2["nu0"][100_000] = np.nan
    with pytest.raises(M.MarfaError) as e:
        M.marfa_prepare_lines(bad2, wl.species)
    assert "line 7:" in str(e.value)


def _prepare_error(M, lines, species):
    try:
        M.marfa_prepare_lines(lines, species)
    except M.MarfaError as e:
        return str(e)
    return None


def test_prepare_lines_concurrent_callers_share_the_host_pool(M):
    """Two host threads validating large line lists at once: the worker pool runs one
    job at a time, and each caller gets the error of its own input."""
    import threading
    from workloads import config0_tiny
    wl = config0_tiny()
    big = np.resize(wl.lines, 150_000)
    bad = [big.copy() for _ in range(4)]
    for k, b in enumerate(bad):
        b["nu0"][20_000 * (k + 1) + k] = np.nan
    got = [None] * len(bad)

    def run(k):
        for _ in range(5):
            got[k] = _prepare_error(M, bad[k], wl.species)

    th = [threading.Thread(target=run, args=(k,)) for k in range(len(bad))]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=120)
        assert not t.is_alive()
    for k in range(len(bad)):
        assert got[k] is not None and f"line {20_000 * (k + 1) + k}:" in got[k]


def _child_prepare(conn):
    from paper_2411_03418_gb300 import marfa as M
    from workloads import config0_tiny
    wl = config0_tiny()
    bad = np.resize(wl.lines, 120_000)
    bad["nu0"][99_999] = -5.0
    conn.send(_prepare_error(M, bad, wl.species))
    conn.close()


@pytest.mark.filterwarnings("ignore:This process .* is multi-threaded")
def test_prepare_lines_after_fork(M):
    """A child forked after the host pool started (it inherits no pool threads) starts a
    pool of its own instead of waiting on the parent's."""
    import multiprocessing as mp
    import torch
    if torch.cuda.is_available():
        pytest.skip("forking after CUDA initialisation is not supported")
    from workloads import config0_tiny
    wl = config0_tiny()
    first = np.resize(wl.lines, 120_000)
    first["nu0"][50_000] = -1.0
    assert "line 50000:" in _prepare_error(M, first, wl.species)  # the parent's pool is up
    ctx = mp.get_context("fork")
    a, b = ctx.Pipe()
    p = ctx.Process(target=_child_prepare, args=(b,))
    p.start()
    ok = a.poll(120)
    p.join(timeout=30)
    if p.is_alive():
        p.kill()
    assert ok, "the forked child did not finish its line preparation"
    msg = a.recv()
    assert msg is not None and "line 99999:" in msg


def test_pipe_rate_rejects_bad_arguments(M):
    import ctypes
    r = ctypes.c_double(0.0)
    for pipe, out in [(7, ctypes.byref(r)), (-1, ctypes.byref(r)), (0, None)]:
        with pytest.raises(M.MarfaError) as e:
            M._check(M.load().marfa_diag_pipe_rate(pipe, out))
        assert e.value.code == -1


@pytest.mark.parametrize("kind", ["uniform", "ties", "sub_unit", "crowded", "extremes", "sorted", "reversed"])
def test_line_order_is_the_stable_sort_by_nu0(M, kind):
    """The host sort behind marfa_prepare_lines (chunked on the worker pool) equals a
    stable sort by nu0, on inputs that stress its buckets."""
    rng = np.random.default_rng(11)
    n = 300_007
    nu = {
        "uniform": 500.0 + 9000.0 * rng.random(n),
        "ties": 2000.0 + np.floor(rng.random(n) * 40) / 8,
        "sub_unit": 1000.0 + 1e-13 * np.floor(rng.random(n) * 300),   # closer than 2^-43 cm^-1
        "crowded": np.where(rng.random(n) < 0.9, 2300.0 + 1e-3 * rng.random(n), 100.0 + 9e4 * rng.random(n)),
        "extremes": rng.choice(np.array([0.0, -0.0, 1e5, 5e4]), n),
        "sorted": np.sort(500.0 + 9000.0 * rng.random(n)),
        "reversed": np.sort(500.0 + 9000.0 * rng.random(n))[::-1].copy(),
    }[kind]
    lines = np.zeros(n, dtype=M.LINE_DTYPE)
    lines["nu0"] = nu
    order = M.marfa_diag_line_order(lines)
    assert np.array_equal(order, np.argsort(nu, kind="stable"))


def test_line_order_small_inputs(M):
    """Short line lists (below one worker chunk, and around the 32-line insertion-sort
    limit) with ties, in the order of a stable sort by nu0."""
    rng = np.random.default_rng(3)
    for n in list(range(1, 70)) + [127, 128, 129, 1000, 8191, 8193, 16385]:
        lines = np.zeros(n, dtype=M.LINE_DTYPE)
        lines["nu0"] = np.floor(rng.random(n) * max(2, n // 3)) * 0.5 + 1000.0
        assert np.array_equal(M.marfa_diag_line_order(lines), np.argsort(lines["nu0"], kind="stable")), n


def test_fail_alloc_environment_arms_the_injector():
    """MARFA_FAIL_ALLOC=n arms the allocation-failure injector when the library loads
    (checked in a fresh process; no GPU call is made)."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2411_03418_gb300 import marfa as M\n"
            "M.load(); print(M.marfa_diag_fail_alloc(0), M.marfa_diag_fail_alloc(0))" % root)
    env = dict(os.environ, MARFA_FAIL_ALLOC="7")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.split() == ["7", "0"]
