"""Seeded synthetic line lists, PT profiles and requests for the five workloads.

The HITRAN 2020 / HITEMP line lists and the Venus profile files the paper works with
(Sec. 3, Sec. 4.2) are not available here, so every workload is synthetic:

* the line record layout is the 36-byte database record of Appendix B
  (nu0 f64, S296, gamma_air, gamma_self, E'', n_air f32, jointMolIso i32, delta_air f32);
* parameter distributions, PT profiles, windows and cut-offs follow the five
  workload descriptions (tiny / Venus 200k x 60 / batch of 256 / Earth 1.2M x 50 /
  surrogate);
* all randomness is numpy PCG64 seeded by the workload index (plus a user seed).

Nothing here evaluates any part of the absorption method.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Appendix B: 8 parameters, 7 x 4 bytes + 8 bytes = 36 bytes per record, no padding.
LINE_DTYPE = np.dtype(
    [
        ("nu0", "<f8"),
        ("S296", "<f4"),
        ("gamma_air", "<f4"),
        ("gamma_self", "<f4"),
        ("E_lower", "<f4"),
        ("n_air", "<f4"),
        ("mol_iso", "<i4"),
        ("delta_air", "<f4"),
    ]
)
assert LINE_DTYPE.itemsize == 36

# One entry per jointMolIso code present in a line list.
SPECIES_DTYPE = np.dtype(
    [("mol_iso", "<i4"), ("chi_enabled", "<i4"), ("mass_amu", "<f8"), ("q_exp", "<f8")]
)
assert SPECIES_DTYPE.itemsize == 24

CO2 = 21  # molecule 2 (CO2), isotopologue 1
H2O = 11  # molecule 1 (H2O), isotopologue 1


@dataclass
class Workload:
    """One absorption request: lines, species table, PT levels and the window.

    ``vmr`` is [n_levels, n_species]; ``shape``/``chi``/``units`` are strings
    ('voigt' | 'lorentz' | 'doppler' | 'const' | 'quad'; 'none' | 'tonkov';
    'sigma' | 'k_cm1' | 'k_km1').
    """

    name: str
    lines: np.ndarray
    species: np.ndarray
    T: np.ndarray
    p: np.ndarray
    vmr: np.ndarray
    nu_lo: float
    nu_hi: float
    cutoff: float
    shape: str = "voigt"
    chi: str = "none"
    units: str = "k_cm1"
    R_w: int = 8
    R_c: int = 8
    surrogate: int = 0
    stencil: int = 3   # interpolation points per coarse panel: 3 (Sec. 2.4) or 5
    # shape 'user': g(x) sampled at x = k user_xmax / (n - 1) on the Lorentz scaling
    user_shape: np.ndarray | None = None
    user_xmax: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def n_levels(self) -> int:
        return int(len(self.T))

    def with_(self, **kw) -> "Workload":
        d = dict(self.__dict__)
        d.update(kw)
        return Workload(**d)

    def level_subset(self, idx) -> "Workload":
        idx = np.asarray(idx)
        return self.with_(T=self.T[idx].copy(), p=self.p[idx].copy(), vmr=self.vmr[idx].copy())


def _species(entries) -> np.ndarray:
    sp = np.zeros(len(entries), dtype=SPECIES_DTYPE)
    for i, (code, chi, mass, q) in enumerate(entries):
        sp[i] = (code, chi, mass, q)
    return sp


def make_lines(rng: np.random.Generator, centres: np.ndarray, mol_iso: int, e_mean: float) -> np.ndarray:
    """Line parameters with the tiny-workload distributions, at the given centres.

    S296 log-uniform 1e-28..1e-19 cm/molecule, gamma_air U(0.05, 0.10),
    gamma_self U(0.07, 0.12) cm^-1/atm, n_air U(0.6, 0.8), delta_air U(-0.01, 0)
    cm^-1/atm, E'' exponential with the given mean (cm^-1).
    """
    n = len(centres)
    ln = np.zeros(n, dtype=LINE_DTYPE)
    ln["nu0"] = centres
    ln["S296"] = np.exp(rng.uniform(np.log(1e-28), np.log(1e-19), n)).astype(np.float32)
    ln["gamma_air"] = rng.uniform(0.05, 0.10, n).astype(np.float32)
    ln["gamma_self"] = rng.uniform(0.07, 0.12, n).astype(np.float32)
    ln["E_lower"] = rng.exponential(e_mean, n).astype(np.float32)
    ln["n_air"] = rng.uniform(0.6, 0.8, n).astype(np.float32)
    ln["mol_iso"] = mol_iso
    ln["delta_air"] = rng.uniform(-0.01, 0.0, n).astype(np.float32)
    return ln


def venus_profile(n_levels: int = 60):
    """T falling linearly 735 -> 170 K, p log-spaced 92 -> 1e-5 atm."""
    u = np.linspace(0.0, 1.0, n_levels)
    T = 735.0 - (735.0 - 170.0) * u
    p = 92.0 * (1e-5 / 92.0) ** u
    return T, p


def config0_tiny(seed: int = 0) -> Workload:
    """2,000 CO2-like lines in 3975-4035 cm^-1, one level (296 K, 1 atm, pure CO2),
    Voigt, 25 cm^-1 cut-off, no chi, window 4000-4010 cm^-1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.uniform(3975.0, 4035.0, 2000)
    lines = make_lines(rng, centres, CO2, 800.0)
    sp = _species([(CO2, 0, 44.0, 1.25)])
    return Workload(
        name="tiny: 2k lines x 1 level, 4000-4010 cm-1, Voigt, cut-off 25",
        lines=lines, species=sp, T=np.array([296.0]), p=np.array([1.0]),
        vmr=np.ones((1, 1)), nu_lo=4000.0, nu_hi=4010.0, cutoff=25.0,
        shape="voigt", chi="none", units="k_cm1",
    )


def _band_centres(rng: np.random.Generator, n_lines: int, lo: float, hi: float) -> np.ndarray:
    """Band-structured centres: P/R branch combs with 0.8 cm^-1 spacing whose band
    origins cluster in Gaussian envelopes around eight band systems."""
    systems = np.array([1950.0, 2080.0, 2230.0, 2350.0, 2500.0, 2680.0, 2850.0, 3040.0])
    widths = np.array([45.0, 60.0, 50.0, 35.0, 70.0, 55.0, 60.0, 45.0])
    weights = np.array([0.8, 1.0, 1.2, 2.0, 1.0, 0.9, 1.1, 0.7])
    weights = weights / weights.sum()
    out = []
    total = 0
    j = np.arange(1, 101)  # 100 rotational lines per branch
    while total < n_lines:
        s = rng.choice(len(systems), p=weights)
        origin = rng.normal(systems[s], widths[s])
        b = 0.8 * (1.0 + rng.uniform(-0.01, 0.01))  # per-band spacing
        curv = rng.uniform(0.0, 0.002)  # band-head curvature
        r_branch = origin + b * j - curv * j * j * 0.1
        p_branch = origin - b * j - curv * j * j * 0.1
        c = np.concatenate([p_branch, r_branch]) + rng.uniform(-0.02, 0.02, 2 * len(j))
        c = c[(c >= lo) & (c <= hi)]
        out.append(c)
        total += len(c)
    c = np.concatenate(out)[:n_lines]
    return c


def config1_venus(seed: int = 1, n_lines: int = 200_000, n_levels: int = 60) -> Workload:
    """200k CO2-like lines, band-structured over 1875-3125 cm^-1; 60 Venus levels;
    Voigt x Tonkov chi, 125 cm^-1 cut-off; window 2000-3000 cm^-1 (2,048,001 points)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = _band_centres(rng, n_lines, 1875.0, 3125.0)
    lines = make_lines(rng, centres, CO2, 800.0)
    sp = _species([(CO2, 1, 44.0, 1.25)])
    T, p = venus_profile(n_levels)
    vmr = np.full((n_levels, 1), 0.965)
    return Workload(
        name=f"venus: {n_lines // 1000}k CO2 lines x {n_levels} levels, 2000-3000 cm-1, Voigt x Tonkov chi, cut-off 125",
        lines=lines, species=sp, T=T, p=p, vmr=vmr,
        nu_lo=2000.0, nu_hi=3000.0, cutoff=125.0,
        shape="voigt", chi="tonkov", units="k_cm1",
    )


def config2_batch(seed: int = 2, n_req: int = 256):
    """256 uneven requests: window width log-U(1, 50) cm^-1 in 500-5000, line count
    log-U(1k, 50k) with the tiny-workload distributions covering window +- cut-off,
    1-100 levels drawn from the Venus profile, cut-off 25 or 125 at random."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    sp = _species([(CO2, 0, 44.0, 1.25)])
    for r in range(n_req):
        width = float(np.exp(rng.uniform(np.log(1.0), np.log(50.0))))
        nu_lo = float(rng.uniform(500.0, 5000.0 - width))
        nu_hi = nu_lo + width
        cutoff = float(rng.choice([25.0, 125.0]))
        n_lines = int(np.exp(rng.uniform(np.log(1000.0), np.log(50000.0))))
        centres = rng.uniform(nu_lo - cutoff, nu_hi + cutoff, n_lines)
        lines = make_lines(rng, centres, CO2, 800.0)
        n_lev = int(rng.integers(1, 101))
        u = rng.uniform(0.0, 1.0, n_lev)
        T = 735.0 - 565.0 * u
        p = 92.0 * (1e-5 / 92.0) ** u
        out.append(Workload(
            name=f"batch request {r}", lines=lines, species=sp, T=T, p=p,
            vmr=np.full((n_lev, 1), 0.965), nu_lo=nu_lo, nu_hi=nu_hi, cutoff=cutoff,
            shape="voigt", chi="none", units="k_cm1",
        ))
    return out


def config3_earth(seed: int = 3, n_lines: int = 1_200_000, n_levels: int = 50) -> Workload:
    """1.2M lines over 475-3025 cm^-1: 70% H2O-like (M=18, Q ~ T^1.5, E'' mean 1200),
    30% CO2-like; 50 levels 288->210 K, 1->1e-3 atm; H2O vmr 1e-2 -> 1e-6 (log),
    CO2 vmr 4e-4; Voigt, 25 cm^-1 cut-off; window 500-3000 cm^-1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_h2o = int(round(0.7 * n_lines))
    n_co2 = n_lines - n_h2o
    l1 = make_lines(rng, rng.uniform(475.0, 3025.0, n_h2o), H2O, 1200.0)
    l2 = make_lines(rng, rng.uniform(475.0, 3025.0, n_co2), CO2, 800.0)
    lines = np.concatenate([l1, l2])
    lines = lines[rng.permutation(len(lines))]
    sp = _species([(H2O, 0, 18.0, 1.5), (CO2, 0, 44.0, 1.25)])
    u = np.linspace(0.0, 1.0, n_levels)
    T = 288.0 - 78.0 * u
    p = 1.0 * (1e-3) ** u
    vmr = np.stack([1e-2 * (1e-4) ** u, np.full(n_levels, 4e-4)], axis=1)
    return Workload(
        name=f"earth: {n_lines / 1e6:.1f}M H2O+CO2 lines x {n_levels} levels, 500-3000 cm-1, Voigt, cut-off 25",
        lines=lines, species=sp, T=T, p=p, vmr=vmr,
        nu_lo=500.0, nu_hi=3000.0, cutoff=25.0,
        shape="voigt", chi="none", units="k_cm1",
    )


def tiny_workload(seed: int, n_lines: int, nu_lo: float, nu_hi: float, cutoff: float,
                  T=(296.0,), p=(1.0,), shape="voigt", chi="none", units="k_cm1",
                  spread: float | None = None, chi_species: int = 0, R_w: int = 8, R_c: int = 8,
                  stencil: int = 3) -> Workload:
    """A small seeded request: n_lines CO2-like lines spread over window +- spread."""
    rng = np.random.Generator(np.random.PCG64(1000 + seed))
    s = cutoff if spread is None else spread
    centres = rng.uniform(nu_lo - s, nu_hi + s, n_lines)
    lines = make_lines(rng, centres, CO2, 800.0)
    sp = _species([(CO2, chi_species, 44.0, 1.25)])
    T = np.asarray(T, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    return Workload(
        name=f"small seed {seed}", lines=lines, species=sp, T=T, p=p,
        vmr=np.full((len(T), 1), 0.965), nu_lo=nu_lo, nu_hi=nu_hi, cutoff=cutoff,
        shape=shape, chi=chi, units=units, R_w=R_w, R_c=R_c, stencil=stencil,
    )
