"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test ties an oracle function to something other than itself: values the paper
prints (tests/golden), closed forms, an independent numerical integration, invariants,
brute force on tiny inputs, and exactness of the eleven-grid bookkeeping on shapes
that 3-point interpolation reproduces exactly. The last block plants plausible
mistakes in the oracle and checks that a pin fails.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

from oracle import marfa_oracle as O
from workloads import LINE_DTYPE, config0_tiny, tiny_workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "grid_and_tables.txt")


def golden():
    d = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            d[k] = v
    return d


# ------------------------------------------------------------ paper-printed constants
def test_grid_constants_from_paper():
    g = golden()
    # Sec. 2.4 / App. A: 20481 finest nodes per 10 cm^-1 (both ends included)
    assert O.num_points(4000.0, 4010.0) == int(g["fine_nodes_per_10cm"])
    assert O.num_points(10.0, 20.0) == int(g["fine_nodes_per_10cm"])
    # N_i = 10 * 2^(i-1) + 1 nodes of grid i in a 10 cm^-1 interval
    for i, key in ((1, "grid_nodes_1"), (2, "grid_nodes_2"), (10, "grid_nodes_10")):
        nodes = (10 * 2 ** O.FIX_BITS) // O.step_fx(i) + 1
        assert nodes == int(g[key])
    # the finest step is 10 / (N - 1)
    assert 2.0 ** -O.FINE_BITS == 10.0 / (int(g["fine_nodes_per_10cm"]) - 1)
    # App. B record length
    assert LINE_DTYPE.itemsize == int(g["line_record_bytes"])


def test_pt_table_layout_from_paper():
    g = golden()
    assert O.pt_record_number(7564.0) == int(g["record_of_7564"])
    assert O.pt_table_name(1) == g["name_of_level_1"]
    assert O.pt_table_name(65) == g["name_of_level_65"]
    k = np.arange(2 * (O.PT_NT - 1) + 1, dtype=np.float32)
    img = np.frombuffer(O.pt_table_bytes(20.0, 40.0, k), dtype="<f4")
    # records 2 and 3 (1-based) cover [20, 30] and [30, 40]; record 1 is zero-filled
    assert len(img) == 3 * O.PT_NT
    assert np.all(img[:O.PT_NT] == 0)
    assert img[O.PT_NT] == 0.0 and img[2 * O.PT_NT - 1] == 20480.0
    assert img[2 * O.PT_NT] == 20480.0  # shared boundary node repeated
    assert img[-1] == 40960.0


# ------------------------------------------------------------ Voigt closed forms and integral
def test_voigt_doppler_limit():
    x = np.linspace(-6, 6, 97)
    assert np.allclose(O.voigt_K(x, 0.0), np.exp(-x * x), rtol=1e-13, atol=0)


def test_voigt_at_centre_is_erfcx():
    y = np.geomspace(1e-4, 1e3, 60)
    assert np.allclose(O.voigt_K(0.0, y), special.erfcx(y), rtol=1e-13)


@pytest.mark.parametrize("x,y", [(0.3, 0.01), (2.5, 0.2), (4.0, 1e-3), (7.0, 0.5), (1.0, 3.0),
                                 (30.0, 2.0), (0.0, 0.05)])
def test_voigt_matches_direct_integration_of_eq8(x, y):
    # Eq. (8) with t = x + y tan(theta): K = (1/pi) int exp(-(x + y tan th)^2) dth
    f = lambda th: math.exp(-(x + y * math.tan(th)) ** 2)
    th0 = -math.atan(x / y)
    val = (integrate.quad(f, -math.pi / 2, th0, epsabs=0, epsrel=1e-13, limit=400)[0]
           + integrate.quad(f, th0, math.pi / 2, epsabs=0, epsrel=1e-13, limit=400)[0]) / math.pi
    assert O.voigt_K(x, y) == pytest.approx(val, rel=1e-10)


def test_voigt_large_y_is_lorentz():
    x = np.linspace(-50, 50, 41)
    y = 1e4
    assert np.allclose(O.voigt_K(x, y), y / (math.sqrt(math.pi) * (x * x + y * y)), rtol=1e-7)


def test_shapes_peak_values_and_unit_integral():
    gL, aD = 0.07, 0.004
    zero = np.zeros(1, dtype=np.int64)
    fL = O.profile("lorentz", zero, 1.0, gL, aD, False)[0]
    fG = O.profile("doppler", zero, 1.0, gL, aD, False)[0]
    fV = O.profile("voigt", zero, 1.0, gL, aD, False)[0]
    assert fL == pytest.approx(1.0 / (math.pi * gL), rel=1e-14)          # Eq. (4) at centre
    assert fG == pytest.approx(math.sqrt(math.log(2) / math.pi) / aD, rel=1e-14)  # Eq. (5)
    y = math.sqrt(math.log(2)) * gL / aD
    assert fV == pytest.approx(math.sqrt(math.log(2) / math.pi) / aD * special.erfcx(y), rel=1e-12)
    # unit integrals on a fine grid: Lorentz with cut-off c integrates to (2/pi) atan(c / g)
    h = 2.0 ** -14
    d = np.arange(-30 * 2 ** 14, 30 * 2 ** 14 + 1, dtype=np.int64) * (2 ** O.FIX_BITS // 2 ** 14)
    for shape, expect in (("lorentz", 2 / math.pi * math.atan(30 / gL)), ("doppler", 1.0)):
        v = O.profile(shape, d, 1.0, gL, aD, False)
        assert integrate.trapezoid(v, dx=h) == pytest.approx(expect, rel=2e-7)
    v = O.profile("voigt", d, 1.0, gL, aD, False)
    # Voigt tails beyond 30 cm^-1 behave as the Lorentz tails
    assert integrate.trapezoid(v, dx=h) == pytest.approx(2 / math.pi * math.atan(30 / gL), rel=1e-5)


def test_appendix_c_asymptote():
    g = golden()
    x = float(g["voigt_lorentz_x"])
    for y in (1e-3, 1e-2, 0.1):
        K = O.voigt_K(x, y)
        lor = y / (math.sqrt(math.pi) * (x * x + y * y))
        assert abs(K / (lor * (1 + 1.5 / x ** 2)) - 1) < float(g["voigt_asymptote_tolerance"])
        assert abs(K / lor - 1) < float(g["voigt_asymptote_tolerance"])


# ------------------------------------------------------------ spectroscopy
def _one_line(nu0=2349.0, S=1e-20, ga=0.07, gs=0.09, E=500.0, n=0.7, d=-0.003):
    ln = np.zeros(1, dtype=LINE_DTYPE)
    ln[0] = (nu0, S, ga, gs, E, n, 21, d)
    return ln


def _wl_one(T, p, vmr=1.0, units="sigma", **kw):
    wl = tiny_workload(0, 5, 2300.0, 2400.0, 25.0, T=(T,), p=(p,), units=units)
    wl = wl.with_(lines=_one_line(**kw), vmr=np.full((1, 1), vmr))
    return wl


def test_spectroscopy_reference_identities():
    ln = _one_line()
    wl = _wl_one(296.0, 0.7, vmr=0.3)
    P = O.level_params(wl, 0)
    assert P["S_T"][0] == pytest.approx(float(ln["S296"][0]), rel=1e-14)
    assert P["gamma_L"][0] == pytest.approx(float(ln["gamma_air"][0]) * 0.7 * 0.7
                                            + float(ln["gamma_self"][0]) * 0.7 * 0.3, rel=1e-14)
    assert P["nu_shift"][0] == pytest.approx(2349.0 + float(ln["delta_air"][0]) * 0.7, rel=1e-15)
    # Doppler HWHM from SI constants with the atomic mass unit (independent route)
    amu = 1.66053906660e-27
    aD = 2349.0 * math.sqrt(2 * math.log(2) * 1.380649e-23 * 296.0 / (44 * amu)) / 2.99792458e8
    assert P["alpha_D"][0] == pytest.approx(aD, rel=1e-9)
    assert 2.17e-3 < aD < 2.19e-3  # the textbook ~0.0022 cm^-1 of CO2 near 2349 cm^-1


def test_number_density_loschmidt():
    # ideal gas at 296 K and 1 atm: 2.4794e19 molecules/cm^3
    assert O.number_density(1.0, 296.0, 1.0) == pytest.approx(2.4794e19, rel=1e-4)
    wl = _wl_one(296.0, 1.0, units="k_cm1")
    P = O.level_params(wl, 0)
    assert P["amp"][0] == pytest.approx(P["S_T"][0] * 2.4794e19, rel=1e-4)
    wl = _wl_one(296.0, 1.0, units="k_km1")
    assert O.level_params(wl, 0)["amp"][0] == pytest.approx(P["S_T"][0] * 2.4794e24, rel=1e-4)


def test_intensity_temperature_dependence():
    # two lines differing only in E'': ratio follows the Boltzmann factor
    T = 700.0
    wa = _wl_one(T, 1.0, E=0.0)
    wb = _wl_one(T, 1.0, E=1000.0)
    Sa = O.level_params(wa, 0)["S_T"][0]
    Sb = O.level_params(wb, 0)["S_T"][0]
    assert Sb / Sa == pytest.approx(math.exp(-1.4387769 * 1000.0 * (1 / T - 1 / 296.0)), rel=1e-6)
    # E'' = 0 and a high wavenumber: only the partition sum, Q ~ T^1.25
    wc = _wl_one(T, 1.0, E=0.0, nu0=9000.0)
    assert O.level_params(wc, 0)["S_T"][0] == pytest.approx(1e-20 * (296.0 / T) ** 1.25, rel=1e-6)
    # low wavenumber: stimulated emission matters and lowers S at high T
    wd = _wl_one(T, 1.0, E=0.0, nu0=50.0)
    assert O.level_params(wd, 0)["S_T"][0] < 0.9 * 1e-20 * (296.0 / T) ** 1.25
    # width scales with (296/T)^n_air
    g1 = O.level_params(_wl_one(296.0, 1.0), 0)["gamma_L"][0]
    g2 = O.level_params(_wl_one(592.0, 1.0), 0)["gamma_L"][0]
    assert g2 / g1 == pytest.approx(0.5 ** float(np.float32(0.7)), rel=1e-12)


# ------------------------------------------------------------ chi
def test_tonkov_chi_pieces_and_near_continuity():
    F = 2 ** O.FIX_BITS
    d = lambda v: np.array([int(round(v * F))], dtype=np.int64)
    assert O.chi_tonkov(d(0.0))[0] == 1.0
    assert O.chi_tonkov(d(2.999))[0] == 1.0
    # branch 1 includes 3: jump of 1 - 1.084 exp(-0.081) = 3.4e-4 only
    assert abs(O.chi_tonkov(d(3.0))[0] - 1.0) < 4e-4
    assert O.chi_tonkov(d(3.0))[0] < 1.0
    # the three branches nearly join at 150 and 300 cm^-1 (within 2 % of each other)
    for b in (150.0, 300.0):
        lo = O.chi_tonkov(d(b))[0]
        hi = O.chi_tonkov(d(b) + 1)[0]
        assert lo != hi and abs(lo / hi - 1) < 0.02
    # decreasing beyond 3, symmetric in the sign of the offset
    v = O.chi_tonkov(np.arange(3, 600, 7, dtype=np.int64) * F)
    assert np.all(np.diff(v) < 0)
    assert O.chi_tonkov(-d(42.0))[0] == O.chi_tonkov(d(42.0))[0]
    assert 0.33 < O.chi_tonkov(d(42.0))[0] < 0.36


def test_gstar_thresholds():
    for R_c in (4, 8, 16):
        for g in range(1, 11):
            assert O.gstar(np.array([R_c * 2.0 ** (1 - g)]), R_c)[0] == g
            assert O.gstar(np.array([np.nextafter(R_c * 2.0 ** (1 - g), 0)]), R_c)[0] == g + 1
    assert O.gstar(np.array([1e-9]), 8)[0] == 11
    assert O.gstar(np.array([1e3]), 8)[0] == 1


# ------------------------------------------------------------ the core width W that sets g*
def _voigt_hwhm_by_bisection(gL, aD):
    """Half width at half maximum of the Voigt profile, found by root bracketing on
    scipy's own ``voigt_profile`` (Gaussian sigma = alpha_D / sqrt(2 ln 2), Lorentz HWHM
    gamma_L): a route that shares nothing with the oracle's width formula."""
    from scipy.optimize import brentq
    sigma = aD / math.sqrt(2.0 * math.log(2.0))
    half = 0.5 * special.voigt_profile(0.0, sigma, gL)
    top = gL + aD  # the Voigt HWHM never exceeds the sum of the two half widths
    return brentq(lambda d: special.voigt_profile(d, sigma, gL) - half, 0.0, top,
                  xtol=1e-14 * top, rtol=1e-13)


# Olivero & Longbothum (1977) give their width formula to about 0.02 %; over gamma_L /
# alpha_D in [1e-3, 1e3] its largest deviation from the exact half width is 2.36e-4.
HWHM_BAR = 2.5e-4


def test_shape_hwhm_limits():
    """Both limits of the Voigt width are exact forms: no Doppler width leaves the
    Lorentz half width (0.5346 + sqrt(0.2166) = 1.000003), no Lorentz width the Doppler
    half width; the pure shapes take their own half widths."""
    for gL in (1e-4, 0.07, 3.4, 40.0):
        assert float(O.shape_hwhm("voigt", gL, 0.0)) == pytest.approx(gL, rel=1e-5)
        assert float(O.shape_hwhm("lorentz", gL, 0.002)) == gL
    for aD in (1e-4, 2.2e-3, 0.05):
        assert float(O.shape_hwhm("voigt", 0.0, aD)) == aD
        assert float(O.shape_hwhm("doppler", 0.3, aD)) == aD


def test_shape_hwhm_matches_voigt_half_maximum():
    """Between the limits W is the half width of the Voigt profile to the formula's
    published accuracy, over the width ratios of the workloads (Doppler-dominated upper
    levels to collision-dominated lower ones)."""
    for aD in (1e-3, 2.2e-3, 0.05):
        for ratio in np.logspace(-3, 3, 25):
            gL = float(ratio) * aD
            W = float(O.shape_hwhm("voigt", gL, aD))
            ref = _voigt_hwhm_by_bisection(gL, aD)
            assert abs(W / ref - 1.0) <= HWHM_BAR, (gL, aD, W, ref)


def test_shape_hwhm_planted_mistakes_fail(monkeypatch):
    """A mistyped constant or a dropped square in the width formula fails a pin."""
    def planted(a, b, square):
        def W(shape, gL, aD):
            if shape == "lorentz":
                return np.asarray(gL, dtype=np.float64)
            if shape == "doppler":
                return np.asarray(aD, dtype=np.float64)
            d2 = aD * aD if square else aD
            return a * gL + np.sqrt(b * gL * gL + d2)
        return W

    for bad in (planted(0.5436, 0.2166, True), planted(0.5346, 0.2616, True),
                planted(0.5346, 0.2166, False), planted(0.5, 0.25, True)):
        with monkeypatch.context() as m:
            m.setattr(O, "shape_hwhm", bad)
            failed = 0
            for pin in (test_shape_hwhm_limits, test_shape_hwhm_matches_voigt_half_maximum):
                try:
                    pin()
                except AssertionError:
                    failed += 1
            assert failed >= 1


# ------------------------------------------------------------ the fixed-point centre
def test_centre_fixed_rounds_half_to_even():
    """c = rint(nu~0 2^43) rounds a tie to the even neighbour. Near 100 cm^-1 the FP64
    spacing is 2^-46 cm^-1, so centres that fall exactly half-way between two
    fixed-point units exist; the expected integers come from exact rational arithmetic
    (Python's round() of a Fraction rounds half to even)."""
    from fractions import Fraction
    u = 2.0 ** -46
    offs = [4, 12, -4, 20, -12, 1, 3, 5, -5, 0]  # in units of 2^-46: 4 = half a fixed-point unit
    vals = np.array([100.0 + k * u for k in offs], dtype=np.float64)
    want = np.array([round(Fraction(float(v)) * (1 << O.FIX_BITS)) for v in vals], dtype=np.int64)
    got = O.centre_fixed(vals)
    assert np.array_equal(got, want)
    base = 100 << O.FIX_BITS
    # the ties explicitly: +0.5 -> 0, +1.5 -> 2, -0.5 -> 0, +2.5 -> 2, -1.5 -> -2
    assert list(got[:5] - base) == [0, 2, 0, 2, -2]
    # and the same through the pressure shift of a record (nu0 + delta p, Sec. 2.2)
    wl = _wl_one(296.0, 1.0, nu0=100.0, d=3 * 2.0 ** -44)
    c = O.centre_fixed(O.level_params(wl, 0)["nu_shift"])
    assert int(c[0]) - base == 2


def test_centre_fixed_planted_rounding_fails(monkeypatch):
    """Rounding down, or rounding ties away from zero, fails the tie pin."""
    F = float(1 << O.FIX_BITS)
    for bad in (lambda v: np.floor(np.asarray(v) * F).astype(np.int64),
                lambda v: (np.sign(np.asarray(v)) * np.floor(np.abs(np.asarray(v)) * F + 0.5)).astype(np.int64)):
        with monkeypatch.context() as m:
            m.setattr(O, "centre_fixed", bad)
            with pytest.raises(AssertionError):
                test_centre_fixed_rounds_half_to_even()


# ------------------------------------------------------------ eleven-grid bookkeeping
CASES = [
    # T, p, chi, cut-off, R_w, R_c, window
    ((296.0,), (1.0,), "none", 25.0, 8, 8, (1000.0, 1003.3)),
    ((200.0,), (1e-4,), "tonkov", 25.0, 8, 8, (1000.0, 1002.71)),
    ((735.0,), (92.0,), "tonkov", 125.0, 8, 8, (1000.0, 1003.0)),
    ((500.0,), (3.0,), "tonkov", 160.0, 4, 16, (999.13, 1001.0)),
    ((250.0,), (0.05,), "none", 7.3, 16, 4, (1000.0, 1001.5)),
]


@pytest.mark.parametrize("case", CASES)
def test_constant_shape_counts_lines_within_cutoff(case):
    T, p, chi, cut, Rw, Rc, (lo, hi) = case
    wl = tiny_workload(11, 250, lo, hi, cut, T=T, p=p, shape="const", chi=chi, chi_species=1,
                       R_w=Rw, R_c=Rc)
    k = O.eleven_grid(wl, 0)
    P = O.level_params(wl, 0)
    c = O.centre_fixed(P["nu_shift"])
    k_lo, k_hi = O.window_nodes(lo, hi)
    X = np.arange(k_lo, k_hi + 1, dtype=np.int64) << O.fine_shift()
    cut_fx = int(round(cut * O.FIX))
    count = (np.abs(X[:, None] - c[None, :]) <= cut_fx).sum(axis=1)
    assert np.abs(k - count).max() < 1e-9 * max(1, count.max())


@pytest.mark.parametrize("case", CASES)
def test_quadratic_shape_eleven_grid_equals_brute_force(case):
    T, p, chi, cut, Rw, Rc, (lo, hi) = case
    wl = tiny_workload(12, 250, lo, hi, cut, T=T, p=p, shape="quad", chi=chi, chi_species=1,
                       R_w=Rw, R_c=Rc)
    k = O.eleven_grid(wl, 0)
    kb = O.brute_force(wl, 0)
    assert np.abs(k - kb).max() <= 1e-12 * np.abs(kb).max()


# ------------------------------------------------------------ 5-point variant (quartic panels)
def test_lagrange5_reproduces_quartics():
    t = np.linspace(0.0, 4.0, 33)
    w = O.lagrange5(t)
    for p in range(5):
        got = sum(w[j] * float(j) ** p for j in range(5))
        assert np.allclose(got, t ** p, rtol=0, atol=1e-12 * max(1.0, 4.0 ** p))


@pytest.mark.parametrize("case", CASES)
def test_five_point_quartic_shape_equals_brute_force(case):
    """Quartic interpolation on panels of four steps reproduces a quartic exactly, so
    eleven-grid == brute force to round-off proves that the 5-point partition counts
    every finest node once (cut-off edges and chi kinks included)."""
    T, p, chi, cut, Rw, Rc, (lo, hi) = case
    wl = tiny_workload(13, 250, lo, hi, cut, T=T, p=p, shape="quart", chi=chi, chi_species=1,
                       R_w=Rw, R_c=Rc, stencil=5)
    k = O.eleven_grid(wl, 0)
    kb = O.brute_force(wl, 0)
    assert np.abs(k - kb).max() <= 1e-11 * np.abs(kb).max()


def test_three_point_is_not_exact_on_quartics():
    T, p, chi, cut, Rw, Rc, (lo, hi) = CASES[0]
    wl = tiny_workload(13, 250, lo, hi, cut, T=T, p=p, shape="quart", chi=chi, R_w=Rw, R_c=Rc)
    k = O.eleven_grid(wl, 0)
    kb = O.brute_force(wl, 0)
    assert np.abs(k - kb).max() > 1e-6 * np.abs(kb).max()


@pytest.mark.parametrize("case", CASES)
def test_five_point_constant_shape_counts_lines(case):
    T, p, chi, cut, Rw, Rc, (lo, hi) = case
    wl = tiny_workload(11, 250, lo, hi, cut, T=T, p=p, shape="const", chi=chi, chi_species=1,
                       R_w=Rw, R_c=Rc, stencil=5)
    k = O.eleven_grid(wl, 0)
    P = O.level_params(wl, 0)
    c = O.centre_fixed(P["nu_shift"])
    k_lo, k_hi = O.window_nodes(lo, hi)
    X = np.arange(k_lo, k_hi + 1, dtype=np.int64) << O.fine_shift()
    count = (np.abs(X[:, None] - c[None, :]) <= int(round(cut * O.FIX))).sum(axis=1)
    assert np.abs(k - count).max() < 1e-9 * max(1, count.max())


def test_five_point_pointwise_form_agrees(c0):
    c5 = c0.with_(stencil=5)
    k = O.eleven_grid(c5, 0)
    k_lo, _ = O.window_nodes(c5.nu_lo, c5.nu_hi)
    idx = np.array([0, 1, 7, 8, 15, 16, 1023, 4096, 10000, 20479, 20480])
    assert np.allclose(O.eleven_grid_at(c5, 0, k_lo + idx), k[idx], rtol=1e-12, atol=0)


def test_five_point_voigt_error_is_smaller(c0):
    """Sec. 2.4 uses 3-point interpolation; the 5-point variant on four-step panels (same
    partition rules) cuts the interpolation error several-fold at the same R_w, R_c."""
    k_lo, _ = O.window_nodes(c0.nu_lo, c0.nu_hi)
    idx = np.arange(0, 20481, 37)
    kb = O.brute_force(c0, 0, k_lo + idx)
    e3 = np.abs(O.eleven_grid(c0, 0)[idx] / kb - 1).max()
    e5 = np.abs(O.eleven_grid(c0.with_(stencil=5), 0)[idx] / kb - 1).max()
    assert e5 < e3 / 3


def test_five_point_planted_mistake_fails(monkeypatch):
    T, p, chi, cut, Rw, Rc, (lo, hi) = CASES[1]
    wl = tiny_workload(13, 120, lo, hi, cut, T=T, p=p, shape="quart", chi=chi, chi_species=1,
                       R_w=Rw, R_c=Rc, stencil=5)

    def holds():
        k = O.eleven_grid(wl, 0)
        kb = O.brute_force(wl, 0)
        return np.abs(k - kb).max() <= 1e-11 * np.abs(kb).max()

    assert holds()
    with monkeypatch.context() as m:
        orig = O.lagrange5
        m.setattr(O, "lagrange5", lambda t: tuple(reversed(orig(t))))
        assert not holds()


def test_pointwise_form_agrees_with_grid_form(c0):
    k = O.eleven_grid(c0, 0)
    k_lo, _ = O.window_nodes(c0.nu_lo, c0.nu_hi)
    idx = np.array([0, 1, 7, 8, 1023, 4096, 10000, 20479, 20480])
    kp = O.eleven_grid_at(c0, 0, k_lo + idx)
    assert np.allclose(kp, k[idx], rtol=1e-12, atol=0)


def test_voigt_eleven_grid_within_interpolation_error(c0):
    k = O.eleven_grid(c0, 0)
    k_lo, _ = O.window_nodes(c0.nu_lo, c0.nu_hi)
    idx = np.arange(0, 20481, 37)
    kb = O.brute_force(c0, 0, k_lo + idx)
    rel = np.abs(k[idx] / kb - 1)
    # paper (Sec. 2.4): < 1 % at centres, up to ~5 % between lines for its constants;
    # with R_w = R_c = 8 the 3-point scheme stays well inside that
    assert rel.max() < 1e-2
    # tighter constants shrink the interpolation error
    c16 = c0.with_(R_w=16, R_c=16)
    k16 = O.eleven_grid(c16, 0)
    assert np.abs(k16[idx] / kb - 1).max() < rel.max() / 3


def test_tiny_brute_force_single_line_lorentz():
    wl = _wl_one(296.0, 1.0, units="sigma").with_(shape="lorentz", nu_lo=2348.5, nu_hi=2349.5,
                                                 cutoff=0.3)
    kb = O.brute_force(wl, 0)
    P = O.level_params(wl, 0)
    k_lo, k_hi = O.window_nodes(2348.5, 2349.5)
    nu = np.arange(k_lo, k_hi + 1) / 2048.0
    d = nu - P["nu_shift"][0]
    g = P["gamma_L"][0]
    expect = np.where(np.abs(d) <= 0.3, P["S_T"][0] * g / (math.pi * (g * g + d * d)), 0.0)
    assert np.allclose(kb, expect, rtol=1e-12, atol=0)


def test_eval_count_scale(c0):
    st = {}
    O.eleven_grid(c0, 0, stats=st)
    total = sum(st.values())
    # far fewer evaluations than the direct sum over the window (paper: ~100x faster)
    lines_in_reach = 2000
    assert total < lines_in_reach * O.num_points(c0.nu_lo, c0.nu_hi) / 200


# ------------------------------------------------------------ planted mistakes must be caught
def _quad_case():
    T, p, chi, cut, Rw, Rc, (lo, hi) = CASES[1]
    return tiny_workload(12, 120, lo, hi, cut, T=T, p=p, shape="quad", chi=chi, chi_species=1,
                         R_w=Rw, R_c=Rc)


def _quad_pin_holds(wl):
    k = O.eleven_grid(wl, 0)
    kb = O.brute_force(wl, 0)
    return np.abs(k - kb).max() <= 1e-12 * np.abs(kb).max()


def test_planted_mistakes_fail_a_pin(monkeypatch):
    wl = _quad_case()
    assert _quad_pin_holds(wl)
    # 1. transposed interpolation weights
    with monkeypatch.context() as m:
        orig = O.lagrange3
        m.setattr(O, "lagrange3", lambda t: tuple(reversed(orig(t))))
        assert not _quad_pin_holds(wl)
    # 2. ownership that forgets the parent test (double counting)
    with monkeypatch.context() as m:
        m.setattr(O, "owned", lambda g, mm, c, gs, ch, cut, Rw, wide=False: O.accept(g, mm, c, gs, ch, cut, Rw, wide))
        assert not _quad_pin_holds(wl)
    # 3. a wrong sign in the pressure shift breaks the Lorentz single-line pin
    with monkeypatch.context() as m:
        orig_lp = O.level_params

        def bad(wl_, lev):
            P = orig_lp(wl_, lev)
            P["nu_shift"] = 2 * wl_.lines["nu0"] - P["nu_shift"]
            return P
        m.setattr(O, "level_params", bad)
        with pytest.raises(AssertionError):
            test_spectroscopy_reference_identities()
    # 4. support tested on the near edge of a panel instead of the far edge lets
    #    panels straddling the cut-off through: the count pin catches it
    with monkeypatch.context() as m:
        orig_acc = O.accept

        def acc(g, mm, c, gs, ch, cut, Rw, wide=False):
            return orig_acc(g, mm, c, gs, ch, cut + (1 << O.panel_shift(g)), Rw, wide)
        m.setattr(O, "accept", acc)
        with pytest.raises(AssertionError):
            test_constant_shape_counts_lines_within_cutoff(CASES[3])


# ---------------------------------------------------------------- Appendix C: the paper's fast Voigt
def _plane():
    x, y = np.meshgrid(np.linspace(0.0, 40.0, 1601), np.logspace(-4, 2, 97))
    return x.ravel(), y.ravel()


def test_paper_voigt_humlicek_regions_match_faddeeva():
    """Regions I-III (Humlicek's rational approximations), away from the paper's
    substitutions, agree with the Faddeeva function to Humlicek's 1e-4."""
    from scipy.special import wofz
    x, y = _plane()
    keep = (x <= 15) & ~((y < 0.02) & (x > 1) & (x < 5.5)) & ~((x + y < 5.5) & (y < 0.195 * x - 0.176))
    ref = wofz(x[keep] + 1j * y[keep]).real
    got = O.voigt_K_paper(x[keep], y[keep])
    assert np.max(np.abs(got - ref) / ref) < 1e-4


def test_paper_voigt_substitutions():
    """|x| > 15: the Lorentz wing, exactly, within the paper's 1 % of K; region 4: the
    Appendix C asymptote on the Gaussian core, exactly (its error to K, up to about 9 %,
    is the paper's, reported rather than pinned); the rest of Humlicek's region IV (now
    region III's formula) within about 1 % (1.06 % at worst on this grid)."""
    from scipy.special import wofz
    g = golden()
    x, y = _plane()
    ref = wofz(x + 1j * y).real
    got = O.voigt_K_paper(x, y)
    far = x > float(g["voigt_lorentz_x"])
    assert np.allclose(got[far], y[far] / (np.sqrt(np.pi) * (x[far] ** 2 + y[far] ** 2)), rtol=1e-14, atol=0)
    assert np.max(np.abs(got[far] - ref[far]) / ref[far]) < float(g["voigt_asymptote_tolerance"])
    r4 = ((y < float(g["voigt_region4_y_max"])) & (x > float(g["voigt_region4_x_min"]))
          & (x < float(g["voigt_region4_x_max"])))
    k4 = np.exp(-x[r4] ** 2) + y[r4] / (np.sqrt(np.pi) * x[r4] ** 2) * (1 + 1.5 / x[r4] ** 2)
    assert np.allclose(got[r4], k4, rtol=1e-14, atol=0)
    assert 0.05 < np.max(np.abs(got[r4] - ref[r4]) / ref[r4]) < 0.09
    iv = (x + y < 5.5) & (y < 0.195 * x - 0.176) & ~r4
    assert np.max(np.abs(got[iv] - ref[iv]) / ref[iv]) < 0.015
    assert np.array_equal(O.voigt_K_paper(-x, y), got)  # even in x


def test_paper_voigt_profile_normalisation():
    """The 'voigt_paper' shape integrates to 1 like the Voigt profile (to the accuracy of
    its substitutions), by trapezoid on a fine grid out to 400 Doppler widths."""
    gL, aD = 0.003, 0.002
    d = np.linspace(-400 * aD, 400 * aD, 800_001)
    d_fx = np.rint(d * O.FIX).astype(np.int64)
    f = O.profile("voigt_paper", d_fx, 1.0, gL, aD, False)
    g = O.profile("voigt", d_fx, 1.0, gL, aD, False)
    assert abs(np.trapezoid(f, d) / np.trapezoid(g, d) - 1) < 2e-3


# ---------------------------------------------------------------- Sec. 2.2: a user-defined shape
def _lorentz_table(n=200001, x_max=1000.0):
    x = np.linspace(0.0, x_max, n)
    return (1.0 / (1.0 + x * x)).astype(np.float32), x_max


def test_user_shape_of_a_sampled_lorentz_is_the_lorentz_profile():
    """The user's shape g sampled from 1/(1 + x^2) gives Eq. (4) back, within the linear
    interpolation bound max|g''| dx^2 / 8 = dx^2 / 4 near the centre, the float32 rounding
    of the samples, and the (x_max/x)^2 tail's relative error 1/x_max^2 beyond x_max."""
    table, x_max = _lorentz_table()
    dx = x_max / (len(table) - 1)
    gL = 0.07
    d = np.concatenate([np.linspace(0.0, 3.0, 3001), np.linspace(3.0, 200.0, 2001)])
    d_fx = np.round(d * O.FIX).astype(np.int64)
    got = O.profile("user", d_fx, 1.0, gL, 0.002, False, user=(table, x_max))
    ref = O.profile("lorentz", d_fx, 1.0, gL, 0.002, False)
    rel = np.abs(got / ref - 1.0)
    x = d / gL
    bound = (dx * dx / 4.0) * (1.0 + x * x) + 1.2e-7 + np.where(x > x_max, 1.0 / x_max ** 2, 0.0)
    assert np.all(rel <= bound), rel.max()
    # the tail: exactly g(x_max) (x_max / x)^2
    xt = np.array([1500.0, 4000.0])
    assert np.allclose(O.user_g(xt, table, x_max), float(table[-1]) * (x_max / xt) ** 2, rtol=1e-15)


def test_user_shape_interpolates_linearly_and_is_symmetric():
    table = np.array([1.0, 0.5, 0.25, 0.0], np.float32)
    x_max = 3.0
    assert np.allclose(O.user_g([0.0, 0.5, 1.0, 2.5, -2.5], table, x_max), [1.0, 0.75, 0.5, 0.125, 0.125])
    assert O.user_g([3.0], table, x_max)[0] == 0.0


def test_user_shape_planted_scaling_mistake_fails():
    """Scaling the user's g by gamma_L the wrong way (x = d gamma_L) fails the Lorentz pin."""
    table, x_max = _lorentz_table(20001, 100.0)
    d_fx = np.round(np.linspace(0.0, 2.0, 201) * O.FIX).astype(np.int64)
    gL = 0.07
    ref = O.profile("lorentz", d_fx, 1.0, gL, 0.002, False)
    bad = O.user_g(d_fx / O.FIX * gL, table, x_max) / (np.pi * gL)
    assert np.abs(bad / ref - 1.0).max() > 0.5
