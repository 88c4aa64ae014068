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


class _FakeLevels:
    """Three levels: 1000 / 100 / 10 nodes, A_1 with 20 blocks per row."""
    sizes = [(2000, 4 * 27000, 4 * 1000 * 3), (200, 4 * 100 * 20, 4 * 100 * 4), (20, 4 * 100, 0)]

    def amg_num_levels(self, h):
        return 3

    def amg_level_info(self, h, level):
        n, nnz, pnnz = self.sizes[level]
        return dict(n=n, nnz=nnz, n_agg=0, lam=0.0, p_nnz=pnnz)


def test_coarse_levels_roofline_accounting():
    its = 10
    us = {"pre": 40.0, "residual": 30.0, "post1": 50.0, "post2": 40.0}
    bd_ = {f"L1_{k}": (v * its / 1e3, its) for k, v in us.items()}
    bd_.update({"L0_restrict": (20.0 * its / 1e3, its), "L0_prolong": (10.0 * its / 1e3, its),
                "L1_restrict": (5.0 * its / 1e3, its), "L1_prolong": (5.0 * its / 1e3, its)})
    out = bench.coarse_levels_roofline(_FakeLevels(), None, bd_, its, 1000.0, False)
    ops = {e["op"]: e for e in out}
    assert set(ops) == {"A1 (4 smoothing launches)", "R0", "P0", "R1", "P1"}
    a1 = ops["A1 (4 smoothing launches)"]
    assert a1["blocks"] == 2000 and a1["rows"] == 100
    assert a1["us_per_launch"] == pytest.approx(40.0)
    # 36 B per block + row offsets + the mean of 4, 3, 6, 5 vector streams of 16 B
    nbytes = 36 * 2000 + 4 * 101 + 4.5 * 16 * 100
    assert a1["algorithmic_bytes"] == pytest.approx(nbytes)
    assert a1["fp64_ops"] == 4 * 2000
    t_hbm, t_alu = nbytes / 1e12, 8000 / bench.FP64_OPS_PEAK
    assert a1["bound"] == ("alu" if t_alu > t_hbm else "hbm")
    assert a1["frac"] == pytest.approx(max(t_hbm, t_alu) / 40e-6)
    # R0: rows of level 1, P_0's blocks, r gathered over level 0's nodes
    r0 = ops["R0"]
    assert r0["rows"] == 100 and r0["blocks"] == 3000
    assert r0["algorithmic_bytes"] == pytest.approx(36 * 3000 + 4 * 101 + 16 * 1000 + 3 * 16 * 100)
    # the FP32 V-cycle: 20 B per block, 8 B per node and stream, no FP64 operations
    out32 = {e["op"]: e for e in bench.coarse_levels_roofline(_FakeLevels(), None, bd_, its, 1000.0, True)}
    assert out32["P0"]["fp64_ops"] == 0 and out32["P0"]["bound"] == "hbm"
    assert out32["P0"]["algorithmic_bytes"] == pytest.approx(20 * 3000 + 4 * 1001 + 8 * 100 + 2 * 8 * 1000)


def test_csr_equivalent_bandwidth():
    info = {"n": 1000, "nnz": 27000}
    out = bench.csr_equivalent(info, 1e-6, 1000.0, False)
    nbytes = 12 * 27000 + 4 * 1001 + 16 * 1000
    assert out["csr_equivalent_bytes_per_launch"] == nbytes
    assert out["csr_equivalent_gbs"] == pytest.approx(nbytes / 1e-6 / 1e9)
    assert out["csr_equivalent_frac"] == pytest.approx(nbytes / 1e-6 / 1e9 / 1000.0)
    assert bench.csr_equivalent(info, 1e-6, 1000.0, True)["csr_equivalent_bytes_per_launch"] == \
        8 * 27000 + 4 * 1001 + 8 * 1000
    assert bench.csr_equivalent(None, 1e-6, 1000.0, False) == {}
