"""Host-side arithmetic of bench.py, checked without a GPU: the algorithmic
flop count behind the roofline figure, the FP64 peak it is divided by, and
the clock summary that decides whether a timed run is kept."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_host_view", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_stage_flops_of_the_bench_slab():
    """Q = 32, M = 60 (r_cut = 6 sigma at dz = 0.1), m = 10: per velocity
    62 + 64 + 65 + 10 + 6 = 207 flops, per node 896 + 242 + 42 + 100 = 1280,
    so 2 * 32 * 207 + 1280 = 14 528 per node and 59 506 688 per launch on
    the 4096-node slab (the bench line's flops_per_launch)."""
    b = _bench()
    assert b.stage_flops(32, 60, 10) == 14528
    assert b.stage_flops(32, 60, 10) * 4096 == 59506688
    # Q = 16, M = 24, m = 4: per velocity 30 + 32 + 81 = 143, per node
    # 448 + 98 + 18 + 100 = 664
    assert b.stage_flops(16, 24, 4) == 2 * 16 * 143 + 664


def test_fp64_peak_at_the_maximum_clock():
    """152 SMs x 2 FP64 FMA per clock (4 flops) x 2070 MHz = 1258.56 GFLOP/s."""
    b = _bench()
    assert abs(b.fp64_peak_gflops(2070.0) - 1258.56) < 1e-9
    assert abs(b.fp64_peak_gflops(1000.0, sms=1) - 4.0) < 1e-12


def test_clock_summary_reports_median_max_and_active_reasons():
    b = _bench()
    cs = b.ClockSampler()
    assert cs.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
    cs.rows = [
        ["2070", "2070", "900.5", "Not Active", "Not Active", "Not Active", "Active"],
        ["2065", "2070", "950.0", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["1980", "2070", "1010.0", "Not Active", "Active", "Not Active", "Not Active"],
    ]
    s = cs.summary()
    assert s["sm_mhz"] == 2065.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_method_flop_count_of_the_bench_slab():
    """The method's count per node-velocity and stage, 2 (68 + 4Q): 392 at
    Q = 32 (about 1200 per node-velocity-step over the three stages)."""
    import bench as b
    assert b.stage_flops_method(32) == 32 * 392
    assert b.stage_flops_method(16) == 16 * 2 * (68 + 64)
    assert abs(3 * b.stage_flops_method(32) / 32 - 1176) < 1e-12
