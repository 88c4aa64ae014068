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
