"""The MARFA_DEBUG build of the library on the GPU: its kernels check their indexed
accesses and report a failed check through the call's return code (MARFA_E_INTERNAL),
never by trapping. The probe proves that a failing check is caught and reported and the
library stays usable; then the small parity cases run through every kernel variant of
the debug build with no check failing, within 1e-4 of the FP64 oracle. The debug library
runs in a subprocess (the binding holds one library per process)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path.insert(0, ROOT)
import numpy as np
import torch
from paper_2411_03418_gb300 import build, marfa as M
from oracle import marfa_oracle as O
from workloads import tiny_workload

M.load(build.build(debug=True))
assert M.marfa_diag_check(3) is True          # a debug build; in range: no failure
try:
    M.marfa_diag_check(40)                    # out of range: the check fires, no access
    raise SystemExit("the probe's check did not fire")
except M.MarfaError as e:
    assert e.code == -5 and "901" in str(e), e
assert M.marfa_diag_check(5) is True          # cleared and usable again

cases = [
    tiny_workload(61, 400, 2000.0, 2003.01, 125.0, T=(735.0, 296.0, 170.0), p=(92.0, 1.0, 1e-5),
                  chi="tonkov", chi_species=1),
    tiny_workload(62, 300, 1999.13, 2001.0, 400.0, T=(500.0,), p=(0.05,), chi="tonkov", chi_species=1,
                  R_w=4, R_c=16),
    tiny_workload(63, 300, 700.37, 701.9, 7.3, T=(250.0,), p=(0.05,), shape="lorentz"),
    tiny_workload(64, 300, 2000.0, 2001.9, 25.0, T=(296.0, 200.0), p=(1.0, 1e-3), chi="tonkov",
                  chi_species=1, stencil=5),
]
refs = [[O.eleven_grid(w, l) for l in range(w.n_levels)] for w in cases]
for coarse in range(6):
    for fine in range(4):
        v = np.full(11, coarse, np.int32); v[0] = -1; v[10] = fine
        M.marfa_diag_variants(v)
        for w, ref in zip(cases, refs):
            lines = M.marfa_prepare_lines(w.lines, w.species)
            out = np.empty((w.n_levels, M.marfa_num_points(w.nu_lo, w.nu_hi)), np.float32)
            M.marfa_absorption(lines, M.levels_of(w), w.vmr, M.request_of(w), out)
            for l in range(w.n_levels):
                r = ref[l]; mx = np.abs(r).max(); big = np.abs(r) > 1e-8 * mx
                rel = np.abs(out[l][big] / r[big] - 1).max()
                assert rel < 1e-4, (coarse, fine, l, rel)
# a captured, autotuned plan through the debug kernels
w = cases[0]
lines = M.marfa_prepare_lines(w.lines, w.species)
dev = torch.empty((w.n_levels, M.marfa_num_points(w.nu_lo, w.nu_hi)), dtype=torch.float32, device="cuda")
plan = M.marfa_plan_create([lines], [M.levels_of(w)], [w.vmr], [M.request_of(w)], [dev], autotune=True)
M.marfa_plan_execute(plan)
torch.cuda.synchronize()
M.marfa_plan_destroy(plan)
print("debug build ok")
""".replace("ROOT", repr(ROOT))


def test_debug_build_checks_report_and_parity():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, "-c", SCRIPT], capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    assert "debug build ok" in r.stdout


def test_ordinary_build_has_no_checks():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_03418_gb300 import build, marfa
    build.build()
    marfa.load()
    assert marfa.marfa_diag_check(40) is False  # compiled out: no check, no store
