"""Host-side pieces of bench.py that feed its JSON line (no GPU)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_is_read_for_every_kernel_class():
    # the roofline's `traffic` comes from the committed ncu summary; a format slip there would
    # silently turn it into null
    for cls in ("col_state", "row_round", "col_phi", "row_final", "col_final"):
        t = bench.traffic_from_profiles(cls)
        assert t is not None and 1e7 < t < 1e9, (cls, t)
    assert bench.traffic_from_profiles("no_such_class") is None


def test_peaks_use_the_measured_file_when_present():
    peak, kind = bench.peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and peak == float(json.load(open(path))["hbm_gbs"])
    else:
        assert kind == "fallback" and peak == bench.FALLBACK_HBM


def test_host_cpu_fields():
    h = bench.host_cpu()
    assert set(h) == {"cpu_model", "host_logical_cores"}
    assert isinstance(h["cpu_model"], str) and h["host_logical_cores"] >= 1


def test_job_rate_counts_every_rank():
    assert bench.job_rate(10, 1, 1000.0) == 10.0
    assert bench.job_rate(10, 4, 2000.0) == 20.0
