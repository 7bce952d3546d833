"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle, on the GPU.

Bars: bit-exact for the integer work (fixed-point centres, g*, ownership of panels
and nodes, evaluation counts); 1e-4 relative on k(nu) wherever k exceeds 1e-8 of the
window maximum, and an absolute floor of 1e-4 * 1e-8 * max below that.
"""
import numpy as np
import pytest

from oracle import marfa_oracle as O
from workloads import config0_tiny, config1_venus, tiny_workload

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


def assert_parity(got, ref, rtol=RTOL, floor=FLOOR, what=""):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape
    mx = np.abs(ref).max()
    big = np.abs(ref) > floor * mx
    if big.any():
        rel = np.abs(got[big] / ref[big] - 1.0)
        i = int(np.argmax(rel))
        assert rel.max() < rtol, f"{what}: max rel err {rel.max():.3e} at {np.nonzero(big)[0][i]}"
    if (~big).any():
        assert np.abs(got[~big] - ref[~big]).max() <= rtol * floor * mx, f"{what}: floor"


def run_gpu(M, wl, device_out=True):
    import torch
    lines = M.marfa_prepare_lines(wl.lines, wl.species)
    rq = M.request_of(wl)
    n = M.marfa_num_points(wl.nu_lo, wl.nu_hi)
    if device_out:
        out = torch.empty((wl.n_levels, n), dtype=torch.float32, device="cuda")
        M.marfa_absorption(lines, M.levels_of(wl), wl.vmr, rq, out, torch.cuda.current_stream())
        torch.cuda.synchronize()
        return out.cpu().numpy()
    out = np.empty((wl.n_levels, n), dtype=np.float32)
    M.marfa_absorption(lines, M.levels_of(wl), wl.vmr, rq, out, None)
    return out


# ------------------------------------------------------------ FP32 Voigt
def test_voigt_fp32_error_map(M):
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(0, 10, 200000), np.exp(rng.uniform(np.log(1e-3), np.log(1e5), 100000)),
                        -rng.uniform(0, 10, 20000)]).astype(np.float32)
    y = np.concatenate([np.exp(rng.uniform(np.log(1e-5), np.log(10), 200000)),
                        np.exp(rng.uniform(np.log(1e-5), np.log(1e4), 100000)),
                        np.exp(rng.uniform(np.log(1e-4), np.log(3), 20000))]).astype(np.float32)
    got = M.marfa_diag_voigt(x, y)
    ref = O.voigt_K(x.astype(np.float64), y.astype(np.float64))
    rel = np.abs(got / ref - 1)
    assert rel.max() < 5e-6, f"max rel err {rel.max():.3e} at x={x[np.argmax(rel)]}, y={y[np.argmax(rel)]}"
    # region boundaries and the pure-Lorentz far wing
    for xb, yb in [(4.5, 1e-3), (4.4999, 0.5), (0.0, 1.0), (8.0, 1e-4), (99.9, 0.1), (0.0, 4.5),
                   (3.0, 0.2499), (3.0, 0.25), (11.99, 0.1), (0.0, 1e-5), (6.4999, 0.2), (0.25, 0.0)]:
        g = M.marfa_diag_voigt(np.array([xb], np.float32), np.array([yb], np.float32))[0]
        assert abs(g / O.voigt_K(np.float32(xb), np.float32(yb)) - 1) < 5e-6


def test_evaluation_cost_classes(M):
    """Per-grid counts by Voigt cost class: they stay within the plain evaluations, both
    table kinds occur (y ~ 0.06 and y ~ 0.6 here), and they vanish for a non-Voigt shape."""
    wl = tiny_workload(61, 250, 2100.0, 2102.0, 25.0, T=(296.0, 200.0), p=(0.002, 0.02))
    lines = M.marfa_prepare_lines(wl.lines, wl.species)
    _, c5 = M.marfa_diag_absorption_counts(lines, M.levels_of(wl), wl.vmr, M.request_of(wl))
    assert c5.shape == (2, 11, 5)
    assert np.all(c5[:, :, 1] == 0)
    assert np.all(c5[:, :, 2] + c5[:, :, 3] + c5[:, :, 4] <= c5[:, :, 0])
    assert c5[0, :, 4].sum() > 0 and c5[1, :, 2].sum() > 0  # small-y at 0.002 atm, 9x9 cells at 0.02 atm
    _, tot = M.marfa_diag_absorption_counted(lines, M.levels_of(wl), wl.vmr, M.request_of(wl))
    assert np.array_equal(tot, c5[:, :, 0])
    wl2 = wl.with_(shape="lorentz")
    _, c5l = M.marfa_diag_absorption_counts(lines, M.levels_of(wl2), wl2.vmr, M.request_of(wl2))
    assert np.all(c5l[:, :, 2:] == 0) and c5l[:, :, 0].sum() > 0


# ------------------------------------------------------------ integer work, bit-exact
LEVEL_CASES = [
    tiny_workload(21, 300, 2000.0, 2003.0, 25.0, T=(735.0, 500.0, 296.0, 200.0, 170.0),
                  p=(92.0, 5.0, 1.0, 1e-2, 1e-5), chi="tonkov", chi_species=1),
]


def test_centres_and_gstar_bit_exact(M):
    wl = LEVEL_CASES[0]
    for R_c in (4, 8, 16):
        w = wl.with_(R_c=R_c)
        lines = M.marfa_prepare_lines(w.lines, w.species)
        c, g, perm = M.marfa_diag_level_lines(lines, M.levels_of(w), w.vmr, M.request_of(w))
        for lev in range(w.n_levels):
            P = O.level_params(w, lev)
            c_ref = O.centre_fixed(P["nu_shift"])
            W = O.shape_hwhm(w.shape, P["gamma_L"], P["alpha_D"])
            g_ref = O.gstar(W, R_c)
            assert np.array_equal(c[lev][perm], c_ref)
            assert np.array_equal(g[lev][perm].astype(np.int64), g_ref)


OWN_CASES = [
    # T, p, chi, cut-off, R_w, R_c, window
    ((296.0,), (1.0,), "none", 25.0, 8, 8, (1000.0, 1003.3)),
    ((200.0,), (1e-4,), "tonkov", 25.0, 8, 8, (1000.0, 1002.71)),
    ((735.0,), (92.0,), "tonkov", 125.0, 8, 8, (1000.0, 1003.0)),
    ((500.0,), (3.0,), "tonkov", 160.0, 4, 16, (999.13, 1001.0)),
    ((250.0,), (0.05,), "none", 7.3, 16, 4, (1000.0, 1001.5)),
]


@pytest.mark.parametrize("case", OWN_CASES)
def test_ownership_bit_exact(M, case):
    T, p, chi, cut, Rw, Rc, (lo, hi) = case
    wl = tiny_workload(31, 200, lo, hi, cut, T=T, p=p, chi=chi, chi_species=1, R_w=Rw, R_c=Rc)
    lines = M.marfa_prepare_lines(wl.lines, wl.species)
    rq = M.request_of(wl)
    _, _, perm = M.marfa_diag_level_lines(lines, M.levels_of(wl), wl.vmr, rq)
    P = O.level_params(wl, 0)
    c = O.centre_fixed(P["nu_shift"])
    gs = O.gstar(O.shape_hwhm(wl.shape, P["gamma_L"], P["alpha_D"]), Rc)
    cut_fx = int(round(cut * O.FIX))
    k_lo, k_hi = O.window_nodes(lo, hi)
    X_lo = k_lo << O.fine_shift()
    for g in range(1, 12):
        if g <= 10:
            s = O.panel_shift(g)
            first = (X_lo >> s) - 300
            count = 800
            m = np.arange(first, first + count, dtype=np.int64)
            ref = np.stack([O.owned(g, m, np.full(count, c[i]), np.full(count, gs[i]),
                                    np.full(count, P["chi_on"][i]), cut_fx, Rw) for i in range(len(c))])
        else:
            first = k_lo - 2000
            count = 4000 + (k_hi - k_lo)
            k = np.arange(first, first + count, dtype=np.int64)
            ref = np.stack([O.fine_owned(k, np.full(count, c[i]), np.full(count, gs[i]),
                                         np.full(count, P["chi_on"][i]), cut_fx, Rw) for i in range(len(c))])
        got = M.marfa_diag_owned(lines, M.levels_of(wl), wl.vmr, rq, 0, g, first, count)
        assert np.array_equal(got[perm].astype(bool), ref), f"grid {g}"


@pytest.mark.parametrize("case", OWN_CASES)
def test_evaluation_counts_match_oracle(M, case):
    T, p, chi, cut, Rw, Rc, (lo, hi) = case
    wl = tiny_workload(41, 300, lo, hi, cut, T=T, p=p, chi=chi, chi_species=1, R_w=Rw, R_c=Rc)
    lines = M.marfa_prepare_lines(wl.lines, wl.species)
    k, counts = M.marfa_diag_absorption_counted(lines, M.levels_of(wl), wl.vmr, M.request_of(wl))
    st = {}
    ref = O.eleven_grid(wl, 0, stats=st)
    assert [int(counts[0][g - 1]) for g in range(1, 12)] == [st[g] for g in range(1, 12)]
    assert_parity(k[0], ref, what="counted run")


# ------------------------------------------------------------ k(nu) parity
PARITY_CASES = [
    dict(seed=51, n=400, lo=1500.0, hi=1504.7, cut=25.0, T=(296.0,), p=(1.0,)),
    dict(seed=52, n=600, lo=2000.0, hi=2003.01, cut=125.0, T=(735.0, 400.0, 170.0), p=(92.0, 0.3, 1e-5),
         chi="tonkov", chi_species=1),
    dict(seed=53, n=300, lo=700.37, hi=701.9, cut=10.0, T=(250.0,), p=(0.02,), shape="lorentz"),
    dict(seed=54, n=300, lo=3000.0, hi=3001.2, cut=5.0, T=(200.0,), p=(1e-4,), shape="doppler"),
    dict(seed=55, n=300, lo=2500.0, hi=2502.0, cut=25.0, T=(296.0,), p=(1.0,), units="sigma"),
    dict(seed=56, n=300, lo=2500.0, hi=2502.0, cut=25.0, T=(220.0,), p=(0.1,), units="k_km1",
         chi="tonkov", chi_species=1),
    dict(seed=57, n=200, lo=1000.0, hi=1000.0 + 1.0 / 2048, cut=3.5, T=(296.0,), p=(1.0,),
         chi="tonkov", chi_species=1),
    # cut-off 400 cm^-1: lines on all three chi branches of Eq. (10) (3-150, 150-300, > 300)
    dict(seed=58, n=400, lo=2000.0, hi=2001.5, cut=400.0, T=(500.0, 250.0), p=(10.0, 0.05),
         chi="tonkov", chi_species=1),
]


@pytest.mark.parametrize("kw", PARITY_CASES)
def test_absorption_parity(M, kw):
    kw = dict(kw)
    wl = tiny_workload(kw.pop("seed"), kw.pop("n"), kw.pop("lo"), kw.pop("hi"), kw.pop("cut"), **kw)
    got = run_gpu(M, wl)
    for lev in range(wl.n_levels):
        assert_parity(got[lev], O.eleven_grid(wl, lev), what=f"level {lev}")


# ------------------------------------------------------------ Appendix C: the paper's fast Voigt
def test_paper_voigt_shape_elementwise(M):
    """The kernels' FP32 paper-mode Voigt against the oracle's FP64 one at the same float32
    points (both choose the region in FP32), every region and its boundaries included.
    Bound: FP32 round-off, largest in region III near the real axis where Re w is a few
    hundred times smaller than |w| (about 5e-5)."""
    xs = np.concatenate([np.linspace(0.0, 40.0, 4001), [1.0, 5.5, 15.0], np.nextafter(np.float32([1.0, 5.5, 15.0]), 0),
                         np.nextafter(np.float32([1.0, 5.5, 15.0]), 100)]).astype(np.float32)
    ys = np.concatenate([np.logspace(-5, 2, 141), [0.02], np.nextafter(np.float32([0.02]), 0)]).astype(np.float32)
    x, y = (a.ravel() for a in np.meshgrid(xs, ys))
    x = np.concatenate([x, -x[:1000]])
    y = np.concatenate([y, y[:1000]])
    got = M.marfa_diag_shape("voigt_paper", x, y).astype(np.float64)
    ref = O.voigt_K_paper(x.astype(np.float64), y.astype(np.float64))
    rel = np.abs(got / ref - 1.0)
    assert rel.max() < 1.5e-4 and np.median(rel) < 1e-6


def test_paper_voigt_absorption(M):
    """The 'voigt_paper' shape through the whole path against the oracle's eleven-grid sum
    with the same shape, at the same 1e-4 bar as the default shape at every node. The
    regions are chosen in FP32 on both sides; a node's x is FP32 on the GPU and FP64 in
    the oracle, so an evaluation within a few roundings of a region boundary could take
    the neighbouring formula; on this case none weighs enough there to move a node by
    1e-4, and every node meets the bar (largest error about 2e-6)."""
    wl = tiny_workload(81, 500, 2000.0, 2003.01, 125.0, T=(735.0, 296.0, 170.0), p=(92.0, 1.0, 1e-5),
                       chi="tonkov", chi_species=1, shape="voigt_paper")
    got = run_gpu(M, wl)
    for lev in range(wl.n_levels):
        assert_parity(got[lev], O.eleven_grid(wl, lev), what=f"paper-mode Voigt level {lev}")


# the 5-point variant (quartic interpolation on panels of four steps)
PARITY_CASES_5 = [
    dict(seed=71, n=400, lo=1500.0, hi=1504.7, cut=25.0, T=(296.0,), p=(1.0,)),
    dict(seed=72, n=600, lo=2000.0, hi=2003.01, cut=125.0, T=(735.0, 400.0, 170.0), p=(92.0, 0.3, 1e-5),
         chi="tonkov", chi_species=1),
    dict(seed=73, n=300, lo=700.37, hi=701.9, cut=10.0, T=(250.0,), p=(0.02,), shape="lorentz"),
    dict(seed=74, n=300, lo=1000.0, hi=1002.0, cut=20.0, T=(300.0, 200.0), p=(2.0, 1e-4), shape="quart",
         chi="tonkov", chi_species=1),
    dict(seed=75, n=250, lo=999.13, hi=1001.0, cut=160.0, T=(500.0,), p=(3.0,), shape="const", chi="tonkov",
         chi_species=1, R_w=4, R_c=16),
]


@pytest.mark.parametrize("kw", PARITY_CASES_5)
def test_absorption_parity_five_point(M, kw):
    kw = dict(kw)
    wl = tiny_workload(kw.pop("seed"), kw.pop("n"), kw.pop("lo"), kw.pop("hi"), kw.pop("cut"), stencil=5, **kw)
    got = run_gpu(M, wl)
    for lev in range(wl.n_levels):
        assert_parity(got[lev], O.eleven_grid(wl, lev), what=f"level {lev}")


def test_host_output_equals_device_output(M):
    wl = tiny_workload(61, 300, 2000.0, 2001.5, 25.0, T=(296.0, 200.0), p=(1.0, 1e-3))
    a = run_gpu(M, wl, device_out=True)
    b = run_gpu(M, wl, device_out=False)
    assert np.array_equal(a, b)


def test_constant_shape_counts_lines(M):
    wl = tiny_workload(62, 500, 1000.0, 1004.0, 30.0, T=(400.0, 200.0), p=(10.0, 1e-4), shape="const",
                       chi="tonkov", chi_species=1)
    got = run_gpu(M, wl)
    k_lo, k_hi = O.window_nodes(wl.nu_lo, wl.nu_hi)
    X = np.arange(k_lo, k_hi + 1, dtype=np.int64) << O.fine_shift()
    cut = int(round(wl.cutoff * O.FIX))
    for lev in range(wl.n_levels):
        c = O.centre_fixed(O.level_params(wl, lev)["nu_shift"])
        count = (np.abs(X[:, None] - c[None, :]) <= cut).sum(axis=1)
        assert np.abs(got[lev] - count).max() <= 1e-6 * count.max()


def test_quadratic_shape_matches_brute_force(M):
    wl = tiny_workload(63, 300, 1000.0, 1002.0, 20.0, T=(300.0, 200.0), p=(2.0, 1e-4), shape="quad",
                       chi="tonkov", chi_species=1)
    got = run_gpu(M, wl)
    for lev in range(wl.n_levels):
        assert_parity(got[lev], O.brute_force(wl, lev), rtol=1e-5, what=f"quad level {lev}")


def test_config0_tiny_full_window(M, c0):
    got = run_gpu(M, c0)
    ref = O.eleven_grid(c0, 0)
    assert_parity(got[0], ref, what="config 0")
    # and the eleven-grid scheme itself against the direct sum (paper: < 1 % at centres)
    k_lo, _ = O.window_nodes(c0.nu_lo, c0.nu_hi)
    idx = np.arange(0, len(ref), 97)
    bf = O.brute_force(c0, 0, k_lo + idx)
    assert np.abs(got[0][idx] / bf - 1).max() < 1e-2


def test_batch_equals_single_bit_identical(M):
    import torch
    wls = [tiny_workload(70 + i, 200 + 50 * i, 1000.0 + 7 * i, 1001.3 + 7.5 * i, [25.0, 125.0][i % 2],
                         T=(296.0, 200.0)[: 1 + i % 2], p=(1.0, 1e-3)[: 1 + i % 2]) for i in range(4)]
    singles = [run_gpu(M, w) for w in wls]
    lines = [M.marfa_prepare_lines(w.lines, w.species) for w in wls]
    outs = [torch.empty((w.n_levels, M.marfa_num_points(w.nu_lo, w.nu_hi)), dtype=torch.float32, device="cuda")
            for w in wls]
    M.marfa_absorption_batch(lines, [M.levels_of(w) for w in wls], [w.vmr for w in wls],
                             [M.request_of(w) for w in wls], outs, torch.cuda.current_stream())
    torch.cuda.synchronize()
    for s, o in zip(singles, outs):
        assert np.array_equal(s, o.cpu().numpy())


def test_prepared_order_is_the_stable_sort_by_nu0(M):
    """The host-side sort (chunks on several threads) gives exactly the order of a stable
    sort by nu0: ties, values closer than one fixed-point unit, a crowded band, shuffled."""
    wl = tiny_workload(97, 50, 1000.0, 1003.0, 25.0, T=(296.0,), p=(1.0,))
    rng = np.random.default_rng(5)
    n = 300_001
    big = np.resize(wl.lines, n)
    nu = np.concatenate([
        1000.0 + np.floor(rng.random(n // 3) * 64) / 16,          # many exact ties
        1001.5 + 1e-13 * np.floor(rng.random(n // 3) * 500),       # below one 2^-43 unit apart
        990.0 + 25.0 * rng.random(n - 2 * (n // 3)),              # spread
    ])
    big["nu0"] = nu[rng.permutation(n)]
    lines = M.marfa_prepare_lines(big, wl.species)
    _, _, perm = M.marfa_diag_level_lines(lines, M.levels_of(wl), wl.vmr, M.request_of(wl))
    order = np.argsort(big["nu0"], kind="stable")
    assert np.array_equal(perm[order], np.arange(n))


def test_window_and_permutation_invariance(M):
    wl = tiny_workload(80, 400, 1000.0, 1003.0, 25.0, T=(296.0,), p=(1.0,))
    a = run_gpu(M, wl)[0]
    sub = wl.with_(nu_lo=1001.0 + 37 / 2048, nu_hi=1002.5)
    b = run_gpu(M, sub)[0]
    k0, _ = O.window_nodes(wl.nu_lo, wl.nu_hi)
    k1, k2 = O.window_nodes(sub.nu_lo, sub.nu_hi)
    assert np.allclose(b, a[k1 - k0:k2 - k0 + 1], rtol=2e-6, atol=0)
    perm = np.random.default_rng(0).permutation(len(wl.lines))
    c = run_gpu(M, wl.with_(lines=wl.lines[perm]))[0]
    assert np.array_equal(a, c)


def test_invalid_requests_rejected(M):
    wl = tiny_workload(90, 50, 1000.0, 1001.0, 25.0)
    lines = M.marfa_prepare_lines(wl.lines, wl.species)
    out = np.empty((1, M.marfa_num_points(1000.0, 1001.0)), np.float32)
    bad = [dict(cutoff=0.0), dict(cutoff=2000.0), dict(shape="nope"), dict(R_w=0), dict(R_c=100),
           dict(nu_lo=1001.0, nu_hi=1000.0)]
    for b in bad:
        kw = dict(nu_lo=1000.0, nu_hi=1001.0, cutoff=25.0)
        kw.update(b)
        try:
            rq = M.make_request(kw["nu_lo"], kw["nu_hi"], kw["cutoff"], kw.get("shape", "voigt"),
                                R_w=kw.get("R_w", 8), R_c=kw.get("R_c", 8))
        except KeyError:
            continue
        with pytest.raises(M.MarfaError) as e:
            M.marfa_absorption(lines, M.levels_of(wl), wl.vmr, rq, out)
        assert e.value.code == -1
    with pytest.raises(M.MarfaError):
        M.marfa_absorption(lines, M.make_levels([-5.0], [1.0]), wl.vmr, M.request_of(wl), out)
    with pytest.raises(M.MarfaError):
        M.marfa_absorption(lines, M.levels_of(wl), np.array([[1.5]]), M.request_of(wl), out)


# ------------------------------------------------------------ full-size Venus workload, sampled
def test_config1_venus_full_size_sampled(M):
    import torch
    wl = config1_venus()
    lines = M.marfa_prepare_lines(wl.lines, wl.species)
    n = M.marfa_num_points(wl.nu_lo, wl.nu_hi)
    assert n == 2_048_001
    out = torch.empty((wl.n_levels, n), dtype=torch.float32, device="cuda")
    M.marfa_absorption(lines, M.levels_of(wl), wl.vmr, M.request_of(wl), out, torch.cuda.current_stream())
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    k_lo, _ = O.window_nodes(wl.nu_lo, wl.nu_hi)
    for lev in (0, 17, 35, 50, 59):
        # the floor from the oracle alone: its largest value over the sampled nodes, which
        # include the centre of the line with the highest peak (a lower bound of the
        # level's maximum, so the floor can only be stricter than the definition's)
        P = O.level_params(wl, lev)
        inside = (P["nu_shift"] > wl.nu_lo) & (P["nu_shift"] < wl.nu_hi)
        peak = np.where(inside, P["amp"] / np.maximum(P["alpha_D"], P["gamma_L"]), 0.0)
        kc = int(np.rint(P["nu_shift"][int(np.argmax(peak))] * 2048)) - k_lo
        idx = np.concatenate([[0, n - 1, kc], rng.integers(0, n, 14)])
        ref = O.eleven_grid_at(wl, lev, k_lo + idx)
        got = out[lev, torch.as_tensor(idx, device="cuda")].cpu().numpy()
        refmax = float(np.abs(ref).max())
        big = np.abs(ref) > FLOOR * refmax
        assert np.all(np.abs(got[big] / ref[big] - 1) < RTOL), f"level {lev}"
        assert np.all(np.abs(got[~big] - ref[~big]) <= RTOL * FLOOR * refmax)


def test_wide_window_full_tiles_parity(M):
    # a window spanning several 64 cm^-1 grid-1 tiles, so that interior tiles (where a
    # line can own every panel) are compared at every output node
    wl = tiny_workload(95, 260, 1000.0, 1140.0, 25.0, T=(735.0, 200.0), p=(3.0, 1e-4),
                       chi="tonkov", chi_species=1)
    got = run_gpu(M, wl)
    for lev in range(wl.n_levels):
        assert_parity(got[lev], O.eleven_grid(wl, lev), what=f"wide window level {lev}")


# ------------------------------------------------------------ Sec. 2.2: a user-defined shape
def test_user_shape_parity(M):
    """The user's tabulated shape (here a sub-Lorentzian g = exp(-x/40) / (1 + x^2), given
    as 4001 samples over [0, 400]) through the kernels' shape switch, with the chi-factor
    and two levels, against the oracle's eleven-grid sum with the same definition; and
    the table sampled from 1/(1 + x^2) against the built-in Lorentz shape."""
    x = np.linspace(0.0, 400.0, 4001)
    g = (np.exp(-x / 40.0) / (1.0 + x * x)).astype(np.float32)
    M.marfa_shape_user_set(g, 400.0)
    wl = tiny_workload(97, 300, 1500.0, 1502.3, 25.0, T=(296.0, 200.0), p=(1.0, 0.05), shape="user",
                       chi="tonkov", chi_species=1).with_(user_shape=g, user_xmax=400.0)
    got = run_gpu(M, wl)
    for lev in range(wl.n_levels):
        assert_parity(got[lev], O.eleven_grid(wl, lev), what=f"user shape level {lev}")
    xs = M.marfa_diag_shape("user", np.linspace(0, 500, 101).astype(np.float32), np.zeros(101, np.float32))
    assert np.allclose(xs, O.user_g(np.linspace(0, 500, 101).astype(np.float32), g, 400.0), rtol=2e-6, atol=1e-12)
    # 4096 samples of 1/(1 + x^2) over [0, 64]: linear interpolation within dx^2/4 = 6e-5
    # near the centre, the (64/x)^2 tail within 1/64^2 = 2.4e-4 of the Lorentz wing
    xl = np.linspace(0.0, 64.0, 4096)
    M.marfa_shape_user_set((1.0 / (1.0 + xl * xl)).astype(np.float32), 64.0)
    lor = tiny_workload(98, 200, 1000.0, 1001.0, 10.0, T=(250.0,), p=(0.05,), shape="lorentz")
    a = run_gpu(M, lor)
    b = run_gpu(M, lor.with_(shape="user"))
    assert_parity(b[0], a[0].astype(np.float64), rtol=5e-4, what="user table of the Lorentz vs Lorentz")


def test_user_shape_requires_a_table(M):
    """A shape outside the library's range or a bad table is refused."""
    with pytest.raises(M.MarfaError):
        M.marfa_shape_user_set(np.array([1.0], np.float32), 1.0)
    with pytest.raises(M.MarfaError):
        M.marfa_shape_user_set(np.array([1.0, -1.0], np.float32), 1.0)
    with pytest.raises(M.MarfaError):
        M.marfa_shape_user_set(np.array([1.0, 0.5], np.float32), 0.0)
