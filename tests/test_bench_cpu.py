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
