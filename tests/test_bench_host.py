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
        expect = d[key]["bytes_per_ray_point"] if d[key]["source_hash"] == b.source_hash(key) else None
        assert b.measured_traffic(key) == expect
        assert d[key]["bytes_per_ray_point"] > 0
