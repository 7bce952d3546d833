"""FP64 CPU oracle of MARFA's line-by-line absorption path (arXiv 2411.03418).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this module.
It shares no code, header, table or constant with the CUDA path, and the product path
never calls it.

What it computes, in the paper's order and notation:

* Sec. 2.1, Eqs. (2)-(3): k(nu; p, T) = n(p, T) sum_j S_j(T) f_j(nu - nu0_j), or the
  cross-section sigma without n.
* Sec. 2.2: temperature/pressure scaling of the line parameters (the paper defers to
  HITRAN's definitions; written out in ``level_params``).
* Sec. 2.2, Eqs. (4)-(8): Lorentz, Gauss and Voigt shapes; K(x, y) = Re w(x + iy)
  with w the Faddeeva function (``scipy.special.wofz`` serves as the library step).
* Appendix C: the paper's own fast Voigt (Lorentz wing beyond |x| = 15, a region-4
  asymptote, Humlicek's rational approximations elsewhere), ``voigt_K_paper``.
* Sec. 2.3, Eqs. (9)-(10): the Tonkov chi-factor.
* Sec. 2.4: the eleven-grid scheme (10 coarse grids + the 2^-11 cm^-1 finest grid,
  quadratic 3-point interpolation onto the finest grid), under the partition reading
  documented in ``accept``; plus the brute-force direct sum on the finest grid, which
  is the plain definition the scheme approximates.
* Appendix A: the PT-table file layout.

Parity status: every function is pinned by ``tests/test_oracle_pins.py``; the partition
rule itself (which wing distances go on which grid) is a reading of Sec. 2.4, pinned by
exactness on quadratic shapes and by the line count on the constant shape, not by
MARFA's own constants (those live in a reference the paper cites but does not print).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import wofz

# ---------------------------------------------------------------- constants
T_REF = 296.0                 # K, HITRAN reference temperature
C2 = 1.438776877              # cm K, second radiation constant hc/k (CODATA 2018)
K_B = 1.380649e-23            # J/K
N_A = 6.02214076e23           # 1/mol
C_LIGHT = 2.99792458e8        # m/s
ATM = 101325.0                # Pa
LN2 = math.log(2.0)

FIX_BITS = 43                 # positions in int64 units of 2^-43 cm^-1
FIX = float(2 ** FIX_BITS)
FINE_BITS = 11                # finest step 2^-11 cm^-1 = 10/20480 (Sec. 2.4, App. A)
NGRID = 10                    # coarse grids G1..G10, h_g = 2^(1-g) cm^-1
CHI_BREAKS = (3.0, 150.0, 300.0)  # Eq. (10) piece boundaries, cm^-1


def fine_shift() -> int:
    """Fixed-point units per finest step: 2^(43-11) = 2^32."""
    return FIX_BITS - FINE_BITS


def panel_shift(g: int) -> int:
    """log2 of the panel width on grid g: a panel spans two steps, 2 h_g = 2^(2-g) cm^-1."""
    return FIX_BITS + 2 - g


def step_fx(g: int) -> int:
    """h_g in fixed-point units (g = 1..10)."""
    return 1 << (FIX_BITS + 1 - g)


# ---------------------------------------------------------------- window
def window_nodes(nu_lo: float, nu_hi: float):
    """Finest-grid node indices k with nu_lo <= k 2^-11 <= nu_hi (Sec. 2.4: N = 20481
    nodes per 10 cm^-1, step 10/20480 = 2^-11)."""
    k_lo = math.ceil(nu_lo * 2048.0)
    k_hi = math.floor(nu_hi * 2048.0)
    return k_lo, k_hi


def num_points(nu_lo: float, nu_hi: float) -> int:
    k_lo, k_hi = window_nodes(nu_lo, nu_hi)
    return max(0, k_hi - k_lo + 1)


# ---------------------------------------------------------------- Sec. 2.2 spectroscopy
def number_density(p_atm, T_K, vmr):
    """n = vmr p / (k_B T) in molecules/cm^3 (Sec. 2.1: n from the profile and abundance)."""
    return vmr * p_atm * ATM / (K_B * T_K) * 1e-6


def level_params(wl, lev: int) -> dict:
    """Per-line parameters at level ``lev`` (Sec. 2.2, HITRAN definitions).

    S(T)   = S296 Q(296)/Q(T) exp(-c2 E''/T)/exp(-c2 E''/296)
             (1 - exp(-c2 nu0/T)) / (1 - exp(-c2 nu0/296)),  Q(T)/Q(296) = (T/296)^q
    gamma_L = (296/T)^n_air (gamma_air (p - p_s) + gamma_self p_s),  p_s = vmr p
    nu~0   = nu0 + delta_air p                     (pressure-shifted centre, Eq. (4))
    alpha_D = nu0/c sqrt(2 N_A k_B T ln2 / M)       (Doppler HWHM, Eq. (5))
    amp    = S(T) [n_s]: the factor the shape multiplies (Eqs. (2)-(3)).
    """
    ln = wl.lines
    T = float(wl.T[lev])
    p = float(wl.p[lev])
    codes = wl.species["mol_iso"]
    sidx = np.searchsorted(np.sort(codes), ln["mol_iso"])
    order = np.argsort(codes)
    sidx = order[sidx]
    assert np.all(codes[sidx] == ln["mol_iso"]), "line with unknown species"
    mass = wl.species["mass_amu"][sidx]
    q = wl.species["q_exp"][sidx]
    vmr = np.asarray(wl.vmr[lev], dtype=np.float64)[sidx]

    nu0 = ln["nu0"].astype(np.float64)
    S296 = ln["S296"].astype(np.float64)
    E = ln["E_lower"].astype(np.float64)
    Q_ratio = (T / T_REF) ** q  # Q(T)/Q(296)
    S_T = (S296 / Q_ratio * np.exp(-C2 * E / T) / np.exp(-C2 * E / T_REF)
           * (1.0 - np.exp(-C2 * nu0 / T)) / (1.0 - np.exp(-C2 * nu0 / T_REF)))
    p_s = vmr * p
    gamma_L = (T_REF / T) ** ln["n_air"].astype(np.float64) * (
        ln["gamma_air"].astype(np.float64) * (p - p_s) + ln["gamma_self"].astype(np.float64) * p_s)
    nu_shift = nu0 + ln["delta_air"].astype(np.float64) * p
    alpha_D = nu0 / C_LIGHT * np.sqrt(2.0 * N_A * K_B * T * LN2 / (mass * 1e-3))
    if wl.units == "sigma":
        amp = S_T
    else:
        amp = S_T * number_density(p, T, vmr)
        if wl.units == "k_km1":
            amp = amp * 1e5
    chi_on = (wl.species["chi_enabled"][sidx] != 0) & (wl.chi == "tonkov")
    return dict(S_T=S_T, gamma_L=gamma_L, alpha_D=alpha_D, nu_shift=nu_shift, amp=amp,
                chi_on=chi_on, T=T, p=p)


def centre_fixed(nu_shift) -> np.ndarray:
    """c = rint(nu~0 2^43), round half to even, as int64."""
    return np.rint(np.asarray(nu_shift, dtype=np.float64) * FIX).astype(np.int64)


def shape_hwhm(shape: str, gamma_L, alpha_D):
    """Half width W that sets the finest grid a line's core needs.

    Voigt: Olivero & Longbothum (1977), W = 0.5346 gL + sqrt(0.2166 gL^2 + aD^2);
    Lorentz: gamma_L; Gauss: alpha_D; test shapes use the Voigt width so that they
    exercise the same partition as the Voigt profile.
    """
    if shape in ("lorentz", "user"):
        return np.asarray(gamma_L, dtype=np.float64)
    if shape == "doppler":
        return np.asarray(alpha_D, dtype=np.float64)
    return 0.5346 * gamma_L + np.sqrt(0.2166 * gamma_L * gamma_L + alpha_D * alpha_D)


def gstar(W, R_c: int) -> np.ndarray:
    """Coarsest grid g in 1..10 whose step resolves the core, h_g <= W / R_c; 11 when
    none does (the core then goes on the finest grid)."""
    W = np.asarray(W, dtype=np.float64)
    gs = np.full(W.shape, NGRID + 1, dtype=np.int64)
    for g in range(NGRID, 0, -1):
        thr = R_c * 2.0 ** (1 - g)
        gs = np.where(W >= thr, g, gs)
    return gs


# ---------------------------------------------------------------- Sec. 2.2-2.3 shapes and chi
def voigt_K(x, y):
    """Voigt function K(x, y) of Eq. (8) = Re w(x + iy), w the Faddeeva function."""
    return wofz(np.asarray(x, dtype=np.float64) + 1j * np.asarray(y, dtype=np.float64)).real


def chi_tonkov(d_fx) -> np.ndarray:
    """Tonkov chi-factor, Eq. (10), of |nu - nu~0| given in fixed-point units.

    Branch 1 includes |d| = 3 and |d| = 150; branch 2 includes 300; chi = 1 below 3.
    """
    a = np.abs(np.asarray(d_fx, dtype=np.int64))
    d = a.astype(np.float64) / FIX
    b3 = int(3 * 2 ** FIX_BITS)
    b150 = int(150 * 2 ** FIX_BITS)
    b300 = int(300 * 2 ** FIX_BITS)
    out = np.ones(a.shape, dtype=np.float64)
    m1 = (a >= b3) & (a <= b150)
    m2 = (a > b150) & (a <= b300)
    m3 = a > b300
    out[m1] = 1.084 * np.exp(-0.027 * d[m1])
    out[m2] = 0.208 * np.exp(-0.016 * d[m2])
    out[m3] = 0.025 * np.exp(-0.009 * d[m3])
    return out


# Humlicek (1982) rational approximations of w(z) = exp(-z^2) erfc(-iz) in t = y - i x, for
# regions I (|x| + y >= 15), II (5.5 <= |x| + y < 15) and III (|x| + y < 5.5); Kuntz (1997)
# evaluates the same rational functions' real parts in real arithmetic.
def _humlicek_w(region: int, t):
    if region == 1:
        return t * 0.5641896 / (0.5 + t * t)
    if region == 2:
        u = t * t
        return t * (1.410474 + u * 0.5641896) / (0.75 + u * (3.0 + u))
    num = 16.4955 + t * (20.20933 + t * (11.96482 + t * (3.778987 + t * 0.5642236)))
    den = 16.4955 + t * (38.82363 + t * (39.27121 + t * (21.69274 + t * (6.699398 + t))))
    return num / den


def voigt_K_paper(x, y):
    """K(x, y) as the paper's Appendix C computes it (its "fast" Voigt): the Lorentz wing
    y / (sqrt(pi) (x^2 + y^2)) for |x| > 15; in region 4 = {y < 0.02, 1 < |x| < 5.5} the
    asymptote exp(-x^2) + y / (sqrt(pi) x^2) (1 + 3 / (2 x^2)) (the Lorentz-wing expansion
    of Appendix C plus the Gaussian core it sits on); elsewhere Re of Humlicek's rational
    approximation of the region |x| + y falls in (I >= 15 > II >= 5.5 > III). The region is
    chosen in FP32, the precision of the paper's code; the values are FP64."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    ax = np.abs(x)
    ax32, y32 = ax.astype(np.float32), y.astype(np.float32)
    s32 = (ax32 + y32).astype(np.float32)
    t = y - 1j * ax
    out = np.where(s32 >= np.float32(15.0), _humlicek_w(1, t).real,
                   np.where(s32 >= np.float32(5.5), _humlicek_w(2, t).real, _humlicek_w(3, t).real))
    r4 = (y32 < np.float32(0.02)) & (ax32 > np.float32(1.0)) & (ax32 < np.float32(5.5))
    with np.errstate(divide="ignore", invalid="ignore"):
        k4 = np.exp(-ax * ax) + y / (math.sqrt(np.pi) * ax * ax) * (1.0 + 1.5 / (ax * ax))
        lor = y / (math.sqrt(np.pi) * (ax * ax + y * y))
    out = np.where(r4, k4, out)
    return np.where(ax32 > np.float32(15.0), lor, out)


QUAD_COEF = (1.0, 0.25, 0.0625)  # test shape f = amp (1 + d/4 + d^2/16), d in cm^-1
QUART_COEF = (1.0, 0.25, 0.0625, 0.015625, 0.00390625)  # f = amp sum_j (d/4)^j, j <= 4


def user_g(x, table, x_max):
    """The user-defined shape of Sec. 2.2's redirectable shape function, as the library
    defines it: g(|x|) linear between the samples table[k] at x = k x_max / (n - 1), and
    g(x_max) (x_max / |x|)^2 beyond x_max."""
    ax = np.abs(np.asarray(x, dtype=np.float64))
    t = np.asarray(table, dtype=np.float64)
    xs = np.linspace(0.0, float(x_max), len(t))
    inside = np.interp(np.minimum(ax, x_max), xs, t)
    tail = t[-1] * (float(x_max) / np.maximum(ax, float(x_max))) ** 2
    return np.where(ax < x_max, inside, tail)


def user_of(wl):
    """The (table, x_max) of a workload's user-defined shape, or None."""
    t = getattr(wl, "user_shape", None)
    return None if t is None else (t, wl.user_xmax)


def profile(shape: str, d_fx, amp, gamma_L, alpha_D, chi_on, user=None):
    """amp * f(d) * chi(|d|) at offsets d (fixed point) from the shifted centre.

    f: 'lorentz' Eq. (4); 'doppler' Eq. (5); 'voigt' Eqs. (7)-(8) ('voigt_paper': with
    K computed as Appendix C does, voigt_K_paper); 'user' the user's tabulated g on the
    Lorentz scaling, f = g(d / gamma_L) / (pi gamma_L) (user = (table, x_max)); test shapes
    'const' (f = 1, no amplitude, no chi: k counts lines), 'quad'
    (f = 1 + d/4 + d^2/16, no chi) and 'quart' (f = sum_{j<=4} (d/4)^j, no chi).
    """
    d = np.asarray(d_fx, dtype=np.int64).astype(np.float64) / FIX
    if shape == "const":
        return np.ones_like(d)
    if shape == "quad":
        a0, a1, a2 = QUAD_COEF
        return amp * (a0 + a1 * d + a2 * d * d)
    if shape == "quart":
        a0, a1, a2, a3, a4 = QUART_COEF
        return amp * (a0 + d * (a1 + d * (a2 + d * (a3 + d * a4))))
    if shape == "lorentz":
        f = gamma_L / (np.pi * (gamma_L * gamma_L + d * d))
    elif shape == "user":
        f = user_g(d / gamma_L, user[0], user[1]) / (np.pi * gamma_L)
    elif shape == "doppler":
        f = math.sqrt(LN2 / np.pi) / alpha_D * np.exp(-d * d * LN2 / (alpha_D * alpha_D))
    elif shape in ("voigt", "voigt_paper"):
        x = math.sqrt(LN2) * d / alpha_D
        y = math.sqrt(LN2) * gamma_L / alpha_D
        K = voigt_K(x, y) if shape == "voigt" else voigt_K_paper(x, y)
        f = math.sqrt(LN2 / np.pi) / alpha_D * K
    else:
        raise ValueError(shape)
    f = amp * f
    chi_on = np.broadcast_to(chi_on, d.shape)
    if np.any(chi_on):
        f = np.where(chi_on, f * chi_tonkov(d_fx), f)
    return f


# ---------------------------------------------------------------- brute force (plain definition)
def brute_force(wl, lev: int, k_nodes=None) -> np.ndarray:
    """k(x) = sum over lines with |x - nu~0| <= cut-off of amp f(x - nu~0) at the finest
    nodes x = k 2^-11 of the window (Eqs. (2)-(3) with the cut-off of Sec. 2.4; the
    cut-off test is exact in fixed point). Sums in math.fsum order per node."""
    P = level_params(wl, lev)
    c = centre_fixed(P["nu_shift"])
    cut = int(round(wl.cutoff * FIX))
    if k_nodes is None:
        k_lo, k_hi = window_nodes(wl.nu_lo, wl.nu_hi)
        k_nodes = np.arange(k_lo, k_hi + 1, dtype=np.int64)
    X = np.asarray(k_nodes, dtype=np.int64) << fine_shift()
    out = np.zeros(len(X))
    order = np.argsort(c, kind="stable")
    cs = c[order]
    for i, x in enumerate(X):
        lo = np.searchsorted(cs, x - cut, side="left")
        hi = np.searchsorted(cs, x + cut, side="right")
        sel = order[lo:hi]
        if len(sel) == 0:
            continue
        v = profile(wl.shape, x - c[sel], P["amp"][sel], P["gamma_L"][sel], P["alpha_D"][sel],
                    P["chi_on"][sel], user=user_of(wl))
        out[i] = math.fsum(v)
    return out


# ---------------------------------------------------------------- Sec. 2.4 eleven-grid partition
def accept(g: int, m, c, gs, chi_on, cut: int, R_w: int, wide: bool = False):
    """Whether grid g (1..10) may carry a line on panel m: the closed interval
    [m P, (m+1) P], P = 2 h_g, with its three nodes at 0, h_g, 2 h_g (wide: P = 4 h_g
    and five nodes, the 5-point variant of Sec. 2.4; the same criteria on the wider
    panels).

    Reading of Sec. 2.4 (centre on the finest grid, wings on ever coarser grids):
      support  : the whole panel lies within the cut-off, d_far <= cut-off;
      smooth   : d_near >= R_w h_g (the panel is at least R_w steps from the centre),
                 or g >= g* (h_g <= W / R_c: the grid resolves the whole core);
      kink-free: with chi on, no Eq. (10) piece boundary |d| in {3, 150, 300} lies in
                 the closed panel, so each panel sees one smooth chi branch.
    d_near/d_far are min/max of |x - c| over the closed panel, exact in fixed point.
    Acceptance is inherited by sub-panels, so the owner of each point is unique.
    """
    m = np.asarray(m, dtype=np.int64)
    c = np.asarray(c, dtype=np.int64)
    s = panel_shift(g) + (1 if wide else 0)
    a = m << s
    b = a + (np.int64(1) << s)
    da = np.abs(a - c)
    db = np.abs(b - c)
    d_far = np.maximum(da, db)
    inside = (a <= c) & (c <= b)
    d_near = np.where(inside, 0, np.minimum(da, db))
    ok = d_far <= cut
    ok &= (d_near >= np.int64(R_w) * step_fx(g)) | (np.asarray(gs) <= g)
    chi_on = np.asarray(chi_on)
    if np.any(chi_on):
        kink = np.zeros(ok.shape, dtype=bool)
        for B in CHI_BREAKS:
            Bf = int(B * 2 ** FIX_BITS)
            for sp in (c - Bf, c + Bf):
                kink |= (a <= sp) & (sp <= b)
        ok &= ~(kink & chi_on)
    return ok


def owned(g: int, m, c, gs, chi_on, cut: int, R_w: int, wide: bool = False):
    """Grid g owns panel m for a line when it accepts it and the parent panel on grid
    g-1 (panel m >> 1, panels of the same number of steps) is not accepted; grid 1 owns
    what it accepts."""
    ok = accept(g, m, c, gs, chi_on, cut, R_w, wide)
    if g > 1:
        ok &= ~accept(g - 1, np.asarray(m, dtype=np.int64) >> 1, c, gs, chi_on, cut, R_w, wide)
    return ok


def fine_owned(k, c, gs, chi_on, cut: int, R_w: int, wide: bool = False):
    """The finest grid evaluates node k itself when |x_k - c| <= cut-off and grid 10
    does not accept the panel containing x_k (half-open panels [a, a+P))."""
    k = np.asarray(k, dtype=np.int64)
    X = k << fine_shift()
    within = np.abs(X - np.asarray(c, dtype=np.int64)) <= cut
    m10 = X >> (panel_shift(NGRID) + (1 if wide else 0))
    return within & ~accept(NGRID, m10, c, gs, chi_on, cut, R_w, wide)


def lagrange3(t):
    """Quadratic Lagrange weights for nodes at 0, 1, 2 evaluated at t."""
    t = np.asarray(t, dtype=np.float64)
    return (t - 1.0) * (t - 2.0) * 0.5, t * (2.0 - t), t * (t - 1.0) * 0.5


def lagrange5(t):
    """Quartic Lagrange weights for nodes at 0, 1, 2, 3, 4 evaluated at t: node j gets
    prod_{i != j} (t - i) / (j - i)."""
    t = np.asarray(t, dtype=np.float64)
    out = []
    for j in range(5):
        w = np.ones_like(t)
        for i in range(5):
            if i != j:
                w = w * (t - i) / (j - i)
        out.append(w)
    return tuple(out)


def stencil_of(wl) -> int:
    """Interpolation points per panel: 3 (the paper's quadratic) or 5 (quartic on panels
    of four steps)."""
    st = int(getattr(wl, "stencil", 3))
    if st not in (3, 5):
        raise ValueError(f"stencil {st}")
    return st


def _line_chunks(n, size):
    for s in range(0, n, size):
        yield slice(s, min(n, s + size))


def eleven_grid(wl, lev: int, stats: dict | None = None, dump: dict | None = None,
                chunk_pairs: int = 4_000_000) -> np.ndarray:
    """The eleven-grid result at every finest node of the window (Sec. 2.4).

    Grids 1..10 (steps 2^(1-g) cm^-1, panels of two steps anchored at nu = 0, which
    is the same as the paper's per-10 cm^-1 grids because 2 h_g divides 10) each sum,
    over the lines that own a panel (``owned``), the profile at that panel's three
    nodes into three panel-local values (left, middle, right). The finest grid sums
    the profile at the nodes it owns (``fine_owned``). Each coarse grid's panel
    values are then interpolated (3-point quadratic) onto the finest nodes of that
    panel and all eleven contributions are added.

    ``stats`` receives the exact number of distinct (line, node) profile evaluations
    per grid; ``dump`` the owned panel / node sets per grid as (line, index) arrays.
    """
    P = level_params(wl, lev)
    c = centre_fixed(P["nu_shift"])
    W = shape_hwhm(wl.shape, P["gamma_L"], P["alpha_D"])
    gs = gstar(W, wl.R_c)
    chi_on = P["chi_on"]
    cut = int(round(wl.cutoff * FIX))
    npn = stencil_of(wl)          # nodes per panel
    wide = npn == 5
    k_lo, k_hi = window_nodes(wl.nu_lo, wl.nu_hi)
    npts = k_hi - k_lo + 1
    X_lo = k_lo << fine_shift()
    X_hi = k_hi << fine_shift()
    knodes = np.arange(k_lo, k_hi + 1, dtype=np.int64)
    Xn = knodes << fine_shift()
    out = np.zeros(npts)
    nl = len(c)
    if dump is not None:
        dump["c"] = c.copy()
        dump["gstar"] = gs.copy()

    def f_at(sel, Xv):
        return profile(wl.shape, Xv - c[sel], P["amp"][sel], P["gamma_L"][sel], P["alpha_D"][sel],
                       chi_on[sel], user=user_of(wl))

    for g in range(1, NGRID + 1):
        s = panel_shift(g) + (1 if wide else 0)
        m_first = X_lo >> s
        m_last = X_hi >> s
        npan = m_last - m_first + 1
        V = [np.zeros(npan) for _ in range(npn)]  # the panel's node values, left to right
        n_eval = 0
        dl, dm = [], []
        per = max(1, chunk_pairs // max(npan, 1))
        for sl in _line_chunks(nl, per):
            idx = np.arange(sl.start, sl.stop)
            mm = np.arange(m_first, m_last + 1, dtype=np.int64)
            li = np.repeat(idx, npan)
            mi = np.tile(mm, len(idx))
            own = owned(g, mi, c[li], gs[li], chi_on[li], cut, wl.R_w, wide)
            li = li[own]
            mi = mi[own]
            if len(li) == 0:
                continue
            if dump is not None:
                dl.append(li)
                dm.append(mi)
            # distinct nodes: the npn - 2 inner nodes once per owned panel; the end nodes
            # shared by neighbouring owned panels of the same line.
            own2 = own.reshape(len(idx), npan)
            left_even = own2.copy()
            left_even[:, 1:] |= own2[:, :-1]
            n_eval += (npn - 2) * int(own2.sum()) + int(left_even.sum()) + int(own2[:, -1].sum())
            a = mi << s
            h = np.int64(1) << (s - (npn - 1).bit_length() + 1)  # the grid step h_g
            slot = mi - m_first
            for q in range(npn):
                V[q] += np.bincount(slot, weights=f_at(li, a + q * h), minlength=npan)
        # interpolate this grid's panels onto the finest nodes
        mp = Xn >> s
        h = np.int64(1) << (s - (npn - 1).bit_length() + 1)
        t = (Xn - (mp << s)).astype(np.float64) / float(h)
        w = lagrange5(t) if wide else lagrange3(t)
        j = mp - m_first
        for q in range(npn):
            out += V[q][j] * w[q]
        if stats is not None:
            stats[g] = n_eval
        if dump is not None:
            dump[g] = (np.concatenate(dl) if dl else np.zeros(0, np.int64),
                       np.concatenate(dm) if dm else np.zeros(0, np.int64))
    # finest grid
    n_eval = 0
    fl, fk = [], []
    acc = np.zeros(npts)
    per = max(1, chunk_pairs // max(npts, 1))
    for sl in _line_chunks(nl, per):
        idx = np.arange(sl.start, sl.stop)
        li = np.repeat(idx, npts)
        ki = np.tile(knodes, len(idx))
        own = fine_owned(ki, c[li], gs[li], chi_on[li], cut, wl.R_w, wide)
        li = li[own]
        ki = ki[own]
        if len(li) == 0:
            continue
        n_eval += len(li)
        if dump is not None:
            fl.append(li)
            fk.append(ki)
        acc += np.bincount(ki - k_lo, weights=f_at(li, ki << fine_shift()), minlength=npts)
    out += acc
    if stats is not None:
        stats[NGRID + 1] = n_eval
    if dump is not None:
        dump[NGRID + 1] = (np.concatenate(fl) if fl else np.zeros(0, np.int64),
                           np.concatenate(fk) if fk else np.zeros(0, np.int64))
    return out


def eleven_grid_at(wl, lev: int, k_nodes, line_block: int = 1 << 16) -> np.ndarray:
    """The eleven-grid value at selected finest nodes, point by point.

    For a node x and a line, the panels containing x on grids 1..10 nest; the coarsest
    grid that accepts its panel owns x for that line and contributes the quadratic
    through the profile at that panel's three nodes; if none accepts and x is within
    the cut-off, the finest grid contributes the profile at x. This is the same sum as
    ``eleven_grid`` (each finest node is covered exactly once per line), evaluated one
    node at a time so that large workloads can be sampled.
    """
    P = level_params(wl, lev)
    c_all = centre_fixed(P["nu_shift"])
    W = shape_hwhm(wl.shape, P["gamma_L"], P["alpha_D"])
    gs_all = gstar(W, wl.R_c)
    chi_all = P["chi_on"]
    cut = int(round(wl.cutoff * FIX))
    npn = stencil_of(wl)
    wide = npn == 5
    order = np.argsort(c_all, kind="stable")
    cs = c_all[order]
    res = np.zeros(len(k_nodes))
    for ii, k in enumerate(np.asarray(k_nodes, dtype=np.int64)):
        X = int(k) << fine_shift()
        lo = np.searchsorted(cs, X - cut, side="left")
        hi = np.searchsorted(cs, X + cut, side="right")
        sel_all = order[lo:hi]
        parts = []
        for s0 in range(0, len(sel_all), line_block):
            sel = sel_all[s0:s0 + line_block]
            c = c_all[sel]
            gs = gs_all[sel]
            ch = chi_all[sel]
            done = np.zeros(len(sel), dtype=bool)
            for g in range(1, NGRID + 1):
                s = panel_shift(g) + (1 if wide else 0)
                m = np.full(len(sel), X >> s, dtype=np.int64)
                acc = accept(g, m, c, gs, ch, cut, wl.R_w, wide) & ~done
                if np.any(acc):
                    j = np.nonzero(acc)[0]
                    a = m[j] << s
                    h = np.int64(1) << (s - (npn - 1).bit_length() + 1)
                    t = float(X - (int(X >> s) << s)) / float(h)
                    w = lagrange5(t) if wide else lagrange3(t)
                    sj = sel[j]
                    fv = [profile(wl.shape, a + q * h - c[j], P["amp"][sj], P["gamma_L"][sj],
                                  P["alpha_D"][sj], ch[j], user=user_of(wl)) for q in range(npn)]
                    parts.append(sum(fv[q] * w[q] for q in range(npn)))
                    done |= acc
            rest = np.nonzero(~done)[0]
            if len(rest):
                sj = sel[rest]
                parts.append(profile(wl.shape, X - c[rest], P["amp"][sj], P["gamma_L"][sj],
                                     P["alpha_D"][sj], ch[rest], user=user_of(wl)))
        res[ii] = math.fsum(np.concatenate(parts)) if parts else 0.0
    return res


def eleven_grid_all(wl) -> np.ndarray:
    """[levels, npts] eleven-grid result for every level."""
    return np.stack([eleven_grid(wl, lev) for lev in range(wl.n_levels)])


# ---------------------------------------------------------------- Appendix A PT-table
PT_NT = 20481  # values per 10 cm^-1 record, both ends included


def pt_table_name(level_number: int) -> str:
    """Level number left-justified and padded with '_' to three characters, '.ptbin'
    appended (Appendix A: 1__.ptbin, 65_.ptbin)."""
    s = str(int(level_number))
    return s + "_" * max(0, 3 - len(s)) + ".ptbin"


def pt_record_number(nu: float) -> int:
    """recNum = int(nu / 10) (Appendix A: 7564 cm^-1 -> record 756)."""
    return int(nu / 10.0)


def pt_table_bytes(nu_lo: float, nu_hi: float, k) -> bytes:
    """Direct-access file image: record r (1-based) holds the 20481 float32 values on
    [10 r, 10 r + 10], at byte offset (r - 1) * 20481 * 4; records below the first one
    written are zero-filled. nu_lo, nu_hi must be multiples of 10 and k must hold the
    finest nodes of [nu_lo, nu_hi]."""
    k = np.asarray(k, dtype=np.float32)
    r0 = pt_record_number(nu_lo)
    r1 = pt_record_number(nu_hi)
    assert len(k) == (r1 - r0) * (PT_NT - 1) + 1
    img = np.zeros((r1 - 1) * PT_NT, dtype="<f4")
    for r in range(r0, r1):
        seg = k[(r - r0) * (PT_NT - 1):(r - r0) * (PT_NT - 1) + PT_NT]
        img[(r - 1) * PT_NT:r * PT_NT] = seg
    return img.tobytes()
