"""Host-side logic of bench.py that needs no GPU."""
import importlib.util
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def test_clock_records_that_force_a_second_measurement():
    b = _bench()
    ok = {"sm_mhz": 2032.0, "sm_max_mhz": 2032.0, "reasons": [], "samples": 6}
    assert not b.clocks_rejected(ok)
    assert not b.clocks_rejected(None)
    assert not b.clocks_rejected({**ok, "reasons": ["sw_power_cap"], "sm_mhz": 1900.0})
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert b.clocks_rejected({**ok, "reasons": [r]})
    assert b.clocks_rejected({**ok, "sm_mhz": 1400.0})  # well below max, no reason: a lock


def test_traffic_record_is_keyed_on_sources_units_and_variant():
    import json
    b = _bench()
    assert b.traffic_record(-1, 0) is None  # no capture has this unit count
    rec = json.load(open(os.path.join(os.path.dirname(b.__file__), "profiles",
                                      "k_eval_mixed_dram.json")))
    if rec["source_sha1"] == b.kernel_source_sha1():
        u = int(rec["units_per_launch"])
        for r in rec["records"]:
            assert b.traffic_record(u, r["variant"]) == r
            assert r["dram_bytes_per_launch"] == r["dram_read_bytes"] + r["dram_write_bytes"]
        assert b.traffic_record(u, 99) is None  # a variant without a capture
