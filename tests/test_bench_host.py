"""Host logic of bench.py (no GPU): the stored oracle runs it scales the CPU
baseline by, looked up by pair and stopping rule."""
import bench


def test_relative_rule_finds_the_stored_bench_pair_run():
    # the 256 x 256 bench pair (white, seed 1000) at relative KKT 1e-6
    assert bench.oracle_iterations(256, "white", 1000, 1e-6) == 440


def test_absolute_rule_finds_only_absolute_runs():
    # the 64 x 64 shapes pair stored at the absolute KKT rule of Table VI
    assert bench.oracle_iterations(64, "shapes", 6, 1e-6, stop="absolute") == 6750
    # a relative-rule lookup never returns an absolute-rule run, and back
    assert bench.oracle_iterations(64, "shapes", 6, 1e-6) != 6750
    assert bench.oracle_iterations(256, "white", 1000, 1e-6, stop="absolute") is None


def test_unknown_pair_has_no_stored_run():
    assert bench.oracle_iterations(256, "white", 12345, 1e-6) is None


def test_recorded_traffic_only_for_the_source_it_was_taken_on(monkeypatch):
    t = bench.SWEEP_TRAFFIC
    assert len(t["kernels_sha256"]) == 64 and t["bytes_per_launch"] > 0
    monkeypatch.setattr(bench, "kernels_sha", lambda: t["kernels_sha256"])
    assert bench.recorded_traffic(256, "fp32") == t["bytes_per_launch"]
    assert bench.recorded_traffic(512, "fp32") is None
    assert bench.recorded_traffic(256, "fp64") is None
    monkeypatch.setattr(bench, "kernels_sha", lambda: "0" * 64)     # the kernels changed since
    assert bench.recorded_traffic(256, "fp32") is None
