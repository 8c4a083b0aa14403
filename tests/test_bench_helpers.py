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


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun with N > 1 only rank 0 times the oracle; the other ranks print nothing
    and exit 0."""
    import subprocess
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
