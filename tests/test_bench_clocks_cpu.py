"""The clock record of bench.py on CPU: the sampler's rows are parsed per device, the rows
written before the timed region are left out when later rows exist, and the throttle
reasons that were active in any kept row are reported."""
import time

import bench

ROW = "{dev}, {sm}, 2070, 900.0, 0x0, {hw}, Not Active, Not Active, {pc}"


def _write(path, rows):
    path.write_text("\n".join(rows) + "\n")


def test_rows_before_the_timed_region_are_left_out(tmp_path):
    p = tmp_path / "clk.csv"
    _write(p, [ROW.format(dev=0, sm=345, hw="Not Active", pc="Not Active"),
               ROW.format(dev=0, sm=2070, hw="Not Active", pc="Active"),
               ROW.format(dev=0, sm=2070, hw="Not Active", pc="Not Active")])
    c = bench.read_clocks(str(p), 0, skip=1)
    assert c["samples"] == 2 and c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    # an idle reading before the timed steps would have pulled the median down
    assert bench.read_clocks(str(p), 0)["samples"] == 3


def test_short_region_falls_back_to_every_row(tmp_path):
    p = tmp_path / "clk.csv"
    _write(p, [ROW.format(dev=0, sm=2070, hw="Active", pc="Not Active")])
    c = bench.read_clocks(str(p), 0, skip=5)
    assert c["samples"] == 1 and c["reasons"] == ["hw_slowdown"]


def test_rows_of_other_devices_are_ignored(tmp_path):
    p = tmp_path / "clk.csv"
    _write(p, [ROW.format(dev=1, sm=1000, hw="Active", pc="Active"),
               ROW.format(dev=0, sm=2070, hw="Not Active", pc="Not Active")])
    c = bench.read_clocks(str(p), 0)
    assert c["samples"] == 1 and c["sm_mhz"] == 2070.0 and c["reasons"] == []
    assert bench.read_clocks(str(p), 3) is None


def test_sampler_lines_waits_at_most_its_limit(tmp_path):
    p = tmp_path / "none.csv"
    t = time.perf_counter()
    assert bench.sampler_lines(str(p), 0.2) == 0
    assert time.perf_counter() - t < 2.0
    _write(p, [ROW.format(dev=0, sm=2070, hw="Not Active", pc="Not Active")] * 3)
    assert bench.sampler_lines(str(p), 5.0) == 3
