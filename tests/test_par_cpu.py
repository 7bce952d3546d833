"""Appendix B ingestion: HITRAN .par text -> line records (marfa_read_par), on the CPU.

The records are synthetic (seeded values, not HITRAN data) written in the fixed-width
layout of the HITRAN 2004+ format: I2 molecule, A1 isotopologue, F12.6 nu, E10.3 S,
E10.3 A, F5.4 gamma_air, F5.3 gamma_self, F10.4 E'', F4.2 n_air, F8.6 delta_air, then
quantum numbers, uncertainty and reference codes and statistical weights (left blank
here) up to 160 columns. Fortran drops the leading zero of a fraction that would not fit
its field (".0712"), and so does the writer below."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def M():
    from paper_2411_03418_gb300 import build, marfa
    build.build()
    marfa.load()
    return marfa


def f_field(x, w, d):
    s = f"{x:.{d}f}"
    if len(s) > w and s.startswith("0."):
        s = s[1:]
    if len(s) > w and s.startswith("-0."):
        s = "-" + s[2:]
    assert len(s) <= w, (x, w, d)
    return s.rjust(w)


def par_record(mol, iso, nu, S, ga, gs, E, n, d):
    rec = (f"{mol:2d}{iso}{f_field(nu, 12, 6)}{S:10.3E}{1.0e-3:10.3E}{f_field(ga, 5, 4)}{f_field(gs, 5, 3)}"
           f"{f_field(E, 10, 4)}{f_field(n, 4, 2)}{f_field(d, 8, 6)}")
    assert len(rec) == 67
    return rec + " " * (160 - 67)


def synthetic(n, seed=0):
    rng = np.random.default_rng(seed)
    rows = []
    for _ in range(n):
        mol = int(rng.integers(1, 13))
        iso = "123456789" [int(rng.integers(0, 9))]
        rows.append((mol, iso, float(rng.uniform(10, 5000)), float(10 ** rng.uniform(-30, -19)),
                     float(rng.uniform(0.01, 0.12)), float(rng.uniform(0.05, 0.5)), float(rng.uniform(0, 5000)),
                     float(rng.uniform(0.3, 0.9)), float(rng.uniform(-0.02, 0.005))))
    return rows


def test_round_trip(M):
    rows = synthetic(300)
    text = "\n".join(par_record(*r) for r in rows).encode() + b"\n"
    got = M.marfa_read_par(text)
    assert len(got) == len(rows)
    for g, (mol, iso, nu, S, ga, gs, E, n, d) in zip(got, rows):
        assert g["mol_iso"] == 100 * mol + int(iso)
        assert g["nu0"] == float(f"{nu:.6f}")
        assert g["S296"] == np.float32(float(f"{S:.3E}"))
        assert g["gamma_air"] == np.float32(round(ga, 4))
        assert g["gamma_self"] == np.float32(round(gs, 3))
        assert g["E_lower"] == np.float32(round(E, 4))
        assert g["n_air"] == np.float32(round(n, 2))
        assert g["delta_air"] == np.float32(round(d, 6))


def test_isotopologue_codes_line_endings_and_blank_lines(M):
    recs = [par_record(2, "0", 2000.0, 1e-21, 0.07, 0.09, 100.0, 0.7, -0.001),
            par_record(2, "A", 2000.5, 2e-21, 0.07, 0.09, 100.0, 0.7, -0.001),
            par_record(12, "B", 2001.0, 3e-21, 0.07, 0.09, 100.0, 0.7, -0.001)]
    text = ("\r\n".join(recs) + "\r\n\r\n   \n").encode()
    got = M.marfa_read_par(text)
    assert list(got["mol_iso"]) == [210, 211, 1212]
    assert list(got["nu0"]) == [2000.0, 2000.5, 2001.0]


def test_count_only_and_errors(M):
    import ctypes
    rows = synthetic(5, seed=1)
    text = "\n".join(par_record(*r) for r in rows).encode()
    lib = M.load()
    n = ctypes.c_int64(-1)
    assert lib.marfa_read_par(text, len(text), None, 0, ctypes.byref(n)) == 0 and n.value == 5
    small = np.zeros(3, dtype=M.LINE_DTYPE)
    assert lib.marfa_read_par(text, len(text), small.ctypes.data, 3, ctypes.byref(n)) < 0
    assert n.value == 5 and np.all(small["nu0"] == 0)  # nothing written
    bad = text + b"\n 2" + b"1" + b"x" * 40 + b"\n"
    with pytest.raises(M.MarfaError, match="line 6"):
        M.marfa_read_par(bad)
    garbled = par_record(*rows[0]).replace(".", ",", 1).encode()
    with pytest.raises(M.MarfaError, match="line 1"):
        M.marfa_read_par(garbled)


def test_records_feed_the_absorption_input(M):
    """Parsed records are the Appendix B structure marfa_prepare_lines takes."""
    got = M.marfa_read_par("\n".join(par_record(*r) for r in synthetic(10, seed=2)).encode())
    assert got.dtype == M.LINE_DTYPE and got.dtype.itemsize == 36
