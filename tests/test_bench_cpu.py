"""CPU checks of bench.py's host-side arithmetic."""
import pytest


def test_wpart_costs_from_kernel_times():
    import bench
    # 2 steps; 1,000 Out elements (8,000 points) + 2,000 sub-cell points in 0.02 + 0.01 ms per step,
    # 500 surface points in 0.005 ms per step
    prof = {"out_elements": (0.04, 2), "cut_elements": (0.02, 2), "nitsche": (0.01, 4)}
    info = {"n_out": 1000, "n_cut_points": 2000, "n_surface_points": 500}
    w = bench.wpart_costs(prof, 2, info)
    assert w["T_v_ps"] == pytest.approx(0.03 / 10000 * 1e9)       # 3,000 ps
    assert w["T_s_ps"] == pytest.approx(0.005 / 500 * 1e9)        # 10,000 ps
    assert w["T_s_over_T_v"] == pytest.approx(10.0 / 3.0)
    assert w["T_out_point_ps"] == pytest.approx(0.02 / 8000 * 1e9)
    assert bench.wpart_costs(prof, 2, dict(info, n_surface_points=0)) is None


def test_clock_summary_reads_only_the_timed_window(tmp_path):
    """Samples written before the start mark (idle clocks) and after the end mark are left out;
    a timed region shorter than one sampling interval falls back to the first sample after it."""
    import bench
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    c.proc = object()        # stands for a running sampler
    row = "0, {}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, {}\n"
    before = row.format(1200, "Not Active")
    inside = row.format(2070, "Not Active") + row.format(2055, "Active")
    after = row.format(1500, "Not Active")
    with open(c.path, "w") as f:
        f.write(before + inside + after)
    c.marks = [len(before), len(before) + len(inside)]
    s = c.summary()
    assert s["samples"] == 2 and s["sm_mhz"] == pytest.approx(2062.5) and s["sm_mhz_min"] == 2055
    assert s["reasons"] == ["sw_power_cap"] and s["window"].startswith("samples written during")
    c.marks = [len(before), len(before)]
    s = c.summary()
    assert s["samples"] == 1 and s["sm_mhz"] == 2070 and s["window"].startswith("timed region shorter")
