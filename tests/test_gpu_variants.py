"""Every summation-kernel variant against the FP64 oracle (GPU).

Grids 2..10 have six kernels (line-major over 32 or 16 node pairs, two-phase,
flattened, by mechanism in a pass per mechanism or one merged pass) and the finest grid
four (8-lane groups per G10 panel, flattened jobs, flattened jobs by mechanism in passes
or merged); a captured plan's autotuner picks one per
grid. The mechanism kernels apply where centre, edges and breakpoints lie apart (the
5-point case below falls back to the general kernels). Each computes the same partition in its
own summation order, so each is held to the same bars: the exact evaluation count per
grid of the oracle (integer), and k(nu) within 1e-4 of the oracle's eleven-grid sum.
The variants are forced through the process-wide defaults (marfa_diag_variants), which
the test restores.
"""
import numpy as np
import pytest

from oracle import marfa_oracle as O
from workloads import tiny_workload

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
    saved = marfa.marfa_diag_variants()
    yield marfa
    marfa.marfa_diag_variants(saved)


def _force(M, coarse, fine):
    v = np.full(11, coarse, dtype=np.int32)
    v[0] = -1
    v[10] = fine
    M.marfa_diag_variants(v)
    assert list(M.marfa_diag_variants()[1:]) == [coarse] * 9 + [fine]


def assert_parity(got, ref, what):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    mx = np.abs(ref).max()
    big = np.abs(ref) > FLOOR * mx
    rel = np.abs(got[big] / ref[big] - 1.0)
    assert rel.max() < RTOL, f"{what}: max rel err {rel.max():.3e}"
    if (~big).any():
        assert np.abs(got[~big] - ref[~big]).max() <= RTOL * FLOOR * mx, f"{what}: floor"


CASES = [
    # Venus-like levels (broad, intermediate and Doppler-narrow lines), chi-factor, 125 cm^-1
    tiny_workload(71, 500, 2000.0, 2003.01, 125.0, T=(735.0, 400.0, 230.0, 170.0), p=(92.0, 0.3, 1e-2, 1e-5),
                  chi="tonkov", chi_species=1),
    # chi on all three branches of Eq. (10), R_w = 4 and R_c = 16, a ragged window
    tiny_workload(72, 400, 1999.13, 2001.0, 400.0, T=(500.0, 250.0), p=(10.0, 0.05), chi="tonkov",
                  chi_species=1, R_w=4, R_c=16),
    # Lorentz and a non-whole cut-off (64-bit ownership form), R_w = 16
    tiny_workload(73, 300, 700.37, 701.9, 7.3, T=(250.0,), p=(0.05,), shape="lorentz", R_w=16, R_c=4),
    # the 5-point partition
    tiny_workload(74, 400, 2000.0, 2001.9, 25.0, T=(296.0, 200.0), p=(1.0, 1e-3), chi="tonkov",
                  chi_species=1, stencil=5),
]


_ORACLE = {}


def _oracle(ci, lev):
    """The oracle's eleven-grid sum and evaluation counts (computed once per case and level)."""
    if (ci, lev) not in _ORACLE:
        st = {}
        _ORACLE[(ci, lev)] = (O.eleven_grid(CASES[ci], lev, stats=st), st)
    return _ORACLE[(ci, lev)]


@pytest.mark.parametrize("coarse", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("fine", [0, 1, 2, 3])
def test_variant_counts_and_parity(M, coarse, fine):
    _force(M, coarse, fine)
    for ci, wl in enumerate(CASES):
        lines = M.marfa_prepare_lines(wl.lines, wl.species)
        k, counts = M.marfa_diag_absorption_counted(lines, M.levels_of(wl), wl.vmr, M.request_of(wl))
        plain = np.empty_like(k)
        M.marfa_absorption(lines, M.levels_of(wl), wl.vmr, M.request_of(wl), plain)
        for lev in range(wl.n_levels):
            ref, st = _oracle(ci, lev)
            assert [int(counts[lev][g - 1]) for g in range(1, 12)] == [st[g] for g in range(1, 12)], \
                f"case {ci} level {lev}: evaluation counts"
            assert_parity(k[lev], ref, f"case {ci} level {lev} (counted)")
            assert_parity(plain[lev], ref, f"case {ci} level {lev}")


def test_variant_constant_shape_counts_lines(M):
    """With f = 1 the result at every node is the exact number of lines within the
    cut-off, whatever the variant (each node gets one contribution per line)."""
    wl = tiny_workload(75, 300, 1500.0, 1502.3, 25.0, T=(735.0, 170.0), p=(92.0, 1e-5), shape="const",
                       chi="tonkov", chi_species=1)
    lines = M.marfa_prepare_lines(wl.lines, wl.species)
    k_lo, k_hi = O.window_nodes(wl.nu_lo, wl.nu_hi)
    X = np.arange(k_lo, k_hi + 1, dtype=np.int64) << O.fine_shift()
    cut_fx = int(round(wl.cutoff * O.FIX))
    for coarse in range(6):
        for fine in range(4):
            _force(M, coarse, fine)
            out = np.empty((wl.n_levels, len(X)), np.float32)
            M.marfa_absorption(lines, M.levels_of(wl), wl.vmr, M.request_of(wl), out)
            for lev in range(wl.n_levels):
                c = O.centre_fixed(O.level_params(wl, lev)["nu_shift"])
                count = (np.abs(X[:, None] - c[None, :]) <= cut_fx).sum(axis=1)
                assert np.abs(out[lev] - count).max() < 1e-3, (coarse, fine, lev)


def test_variants_refuse_out_of_range(M):
    v = M.marfa_diag_variants()
    bad = v.copy()
    bad[3] = 7
    with pytest.raises(M.MarfaError):
        M.marfa_diag_variants(bad)
    assert np.array_equal(M.marfa_diag_variants(), v)
    bad = v.copy()
    bad[10] = 4
    with pytest.raises(M.MarfaError):
        M.marfa_diag_variants(bad)


def test_merged_finest_pass_falls_back_where_an_edge_meets_a_breakpoint(M):
    """A cut-off 1/64 cm^-1 beyond the 150 cm^-1 breakpoint: the mechanisms lie apart
    (mech_fine_ok), but a line's edge and breakpoint fall among one warp's nodes, so the
    finest grid's merged pass does not apply (mech_fine_merge_ok). Forced to the merged
    variant, the library takes the per-mechanism passes and stays within 1e-4 of the
    oracle. A third of the lines sit 150 cm^-1 below the window and a third above, so that
    their edges and breakpoints fall inside it."""
    cut = 150.0 + 1.0 / 64
    base = tiny_workload(76, 600, 2000.0, 2000.5, cut, T=(296.0, 200.0), p=(1.0, 1e-3), chi="tonkov",
                         chi_species=1, spread=0.5)
    ln = base.lines.copy()
    k = len(ln) // 3
    ln["nu0"][:k] -= 150.0
    ln["nu0"][k:2 * k] += 150.0
    wl = base.with_(lines=ln)
    lines = M.marfa_prepare_lines(wl.lines, wl.species)
    refs = [O.eleven_grid(wl, lev) for lev in range(wl.n_levels)]
    for coarse in (2, 4):
        _force(M, coarse, 3)
        out = np.empty((wl.n_levels, M.marfa_num_points(wl.nu_lo, wl.nu_hi)), np.float32)
        M.marfa_absorption(lines, M.levels_of(wl), wl.vmr, M.request_of(wl), out)
        for lev in range(wl.n_levels):
            assert_parity(out[lev], refs[lev], f"coarse {coarse} level {lev}")
