"""Host logic of bench.py: the mode-dependent defaults and the gate on the
recorded ncu traffic (reported only while the kernel sources are unchanged)."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _resolved(*argv):
    return bench.resolve_defaults(bench.parse_args(list(argv)))


def test_time_stepping_defaults():
    a = _resolved()
    assert a.mode == "step" and a.workload == "paper"
    assert a.coarse_eq_limit == bench.STEP_COARSE_EQ_LIMIT
    assert a.autotune == 0                       # the calibrated rule
    assert _resolved("--workload", "large").autotune == 1
    assert _resolved("--autotune", "1").autotune == 1
    assert _resolved("--workload", "large", "--no-autotune").autotune == 0
    assert _resolved("--coarse-eq-limit", "100").coarse_eq_limit == 100


@pytest.mark.parametrize("mode", ["batch", "serve", "sweep"])
def test_other_modes_time_the_forms_and_keep_the_library_coarsening(mode):
    a = _resolved("--mode", mode)
    assert a.autotune == 1 and a.coarse_eq_limit is None


def test_recorded_traffic_only_for_unchanged_sources(monkeypatch):
    kv = {}
    for line in open(bench.TRAFFIC_FILE):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    monkeypatch.setattr(bench, "source_digest", lambda: kv["source_digest"])
    assert bench.recorded_traffic() == float(kv["traffic_bytes_per_launch"])
    assert bench.recorded_traffic(True) == float(kv["traffic_bytes_per_launch_fp32"])
    monkeypatch.setattr(bench, "source_digest", lambda: "0" * 16)
    assert bench.recorded_traffic() is None and bench.recorded_traffic(True) is None


def test_cpu_record_whole_simulation_rate_and_one_core_figure(monkeypatch):
    monkeypatch.setattr(bench, "cpu_model", lambda: "test-cpu")
    r = {"t_setup": 10.0, "t_step": 0.5, "t_step_one_core": 4.0, "iters": [17, 18],
         "threads": 16, "warm": 5, "timed": 20, "one_core_steps": 1}
    c = bench.cpu_record(r, 100)
    assert c["value"] == pytest.approx(100 / (10.0 + 100 * 0.5))
    assert c["cores"] == 16 and c["kind"] == "oracle" and c["cpu_model"] == "test-cpu"
    assert c["one_core"]["value"] == pytest.approx(100 / (10.0 + 100 * 4.0))
    assert c["solve_phase_solves_per_s"] == pytest.approx(2.0)
    assert "time steps 5..24" in c["sample"]
    r["t_step_one_core"] = None
    assert bench.cpu_record(r, 100)["one_core"] is None
