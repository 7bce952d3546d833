"""The two forms of exact panel ownership (csrc/ownership.cuh, rule R2 of Sec. 2.4):
the 32-bit panel-frame masks used by the kernels wherever the cut-off, R_w h_g and the
chi breakpoints are whole panels must equal the 64-bit fixed-point masks bit for bit.
tests/ownership_check.cu draws 400k random and boundary cases (centres on panel ends and
one unit beside them, both parities of the tile's first panel, aligned and unaligned
cut-offs, odd R_w) and compares accept, parent-accept and quick-reject results. Host
code only: built with nvcc, run on the CPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2411_03418_gb300", "csrc")


def test_panel_frame_masks_equal_fixed_point_masks(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "ownership_check")
    build = subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, os.path.join(HERE, "ownership_check.cu"), "-o", exe],
                           capture_output=True, text=True)
    assert build.returncode == 0, build.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    out = run.stdout.strip()
    assert run.returncode == 0, out + "\n" + run.stderr[:4000]
    fields = out.split()
    assert fields[0] == "cases" and fields[4] == "mismatches"
    assert int(fields[5]) == 0
    assert int(fields[3]) > 100000  # enough cases where the frame applies
    assert fields[6] == "mech_cases" and fields[10] == "mech_mismatches"
    assert int(fields[11]) == 0
    assert int(fields[9]) > 20000  # enough cases where the mechanisms act apart
    # the finest grid's merged pass: one edge or breakpoint per warp span where
    # mech_fine_merge_ok holds, and the condition rejects an edge beside a breakpoint
    assert fields[12] == "merge_cases" and int(fields[13]) > 10000
    assert fields[14] == "merge_bad" and int(fields[15]) == 0
    assert fields[16] == "planted" and fields[17] == "1"
