"""Host logic of bench.py that needs no GPU: the roofline traffic figures are
keyed by the formal kernels' code, so that a comment edit keeps them and a
code change voids them."""
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_code_only_drops_comments_and_blank_space():
    b = _bench()
    code = "int a = 1;  // note\n/* block\n comment */\tint b;\n"
    assert b._code_only(code) == "int a = 1; int b;"
    assert b._code_only("x = y / z; // a / b") == "x = y / z;"
    assert b._code_only("p /* x */ q") != b._code_only("pq")


def test_traffic_is_reported_only_for_the_profiled_code():
    b = _bench()
    d = json.load(open(os.path.join(ROOT, "profiles", "formal_traffic.json")))
    for key in b.KERNEL_SOURCES:
        if key not in d:                      # never captured: no traffic figure
            assert b.measured_traffic(key) is None
            continue
        expect = d[key]["bytes_per_ray_point"] if d[key]["source_hash"] == b.source_hash(key) else None
        assert b.measured_traffic(key) == expect
        assert d[key]["bytes_per_ray_point"] > 0


def test_roofline_peaks_from_measured_rates():
    """The roofline of each evaluation kind follows the unit counts and the
    measured pipe rates: FP32-bound for the JVP, MUFU-bound for the value
    evaluation at 128 FP32 lanes against 16 MUFU per clock; FP64 with exp
    costed in FMA-instruction time."""
    b = _bench()
    sm_clk = 152 * 2.07e9
    peaks = {"fp32_fma_per_s": 128 * sm_clk, "mufu_per_s": 16 * sm_clk,
             "fp64_fma_per_s": 1e12, "fp64_exp_per_s": 1e11}
    assert abs(b.peak_rate("jvp", False, peaks) / (sm_clk * 128 / 26) - 1) < 1e-12
    assert abs(b.peak_rate("value", False, peaks) / (sm_clk * 16 / 2) - 1) < 1e-12
    assert abs(b.peak_rate("value", True, peaks) / (1e12 / (10 + 2 * 10)) - 1) < 1e-12
    r = b.kernel_roofline("k", "jvp", False, 1e9, 2.0, 4, peaks)
    assert abs(r["achieved"] - 1e9 / 2e-3 / 1e9) < 1e-9 and abs(r["avg_launch_us"] - 500.0) < 1e-9


def test_stage_breakdown_is_per_active_tick_with_shares():
    b = _bench()
    st = {"formal_launches": 4, "stage_ms": [4.0, 8.0, 2.0, 4.0, 1.0, 1.0]}
    r = b.stage_breakdown(st)
    assert list(r["per_tick"]) == list(b.STAGES)
    assert r["per_tick"]["tangent_sweep"] == 2.0 and r["tick_total"] == 5.0
    assert abs(sum(r["share"].values()) - 1.0) < 1e-12
    assert b.stage_breakdown({"formal_launches": 0, "stage_ms": [0.0] * 6})["tick_total"] == 0.0
