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


def test_traffic_record_is_keyed_on_sources_and_units():
    b = _bench()
    rec = b.traffic_record(-1)  # no capture has this unit count
    assert rec is None
