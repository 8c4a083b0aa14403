"""Host-side pieces of bench.py that feed its JSON line (no GPU)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_table_covers_every_kernel_class_or_is_empty():
    # the roofline's `traffic` comes from a recorded ncu capture of the current kernels; when the
    # table is filled, every class has a plausible per-launch byte count and a named source
    if bench.TRAFFIC_NCU:
        assert bench.TRAFFIC_SOURCE
        for cls in ("col_state", "row_round", "col_phi", "row_final", "col_final"):
            t, src = bench.traffic_of(cls)
            assert t is not None and 1e7 < t < 1e9 and src == bench.TRAFFIC_SOURCE, (cls, t)
    assert bench.traffic_of("no_such_class") == (None, None)


def test_tank_value_ignores_non_finite_runs():
    cases = [{"ms_per_step": 0.2, "state_finite": True}, {"ms_per_step": None, "state_finite": False},
             {"ms_per_step": 0.3, "state_finite": True}]
    assert bench.tank_value(cases) == 0.3
    # a diverged run never sets the value, however long it took
    cases.append({"ms_per_step": 9.9, "state_finite": False})
    assert bench.tank_value(cases) == 0.3
    assert bench.tank_value([{"ms_per_step": 1.0, "state_finite": False}]) is None


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


def test_oracle_threads_is_the_transform_worker_count():
    # the cpu_baseline leg records how many host threads the oracle's transforms use
    n = bench.oracle_threads()
    assert isinstance(n, int) and 1 <= n <= (os.cpu_count() or 1)
