"""Host-side logic of the benchmark (no GPU): the clock sampler's parsing of nvidia-smi lines,
the roofline peaks and their fallback, the kernel classification."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_takes_the_median_and_collects_active_reasons(bench):
    s = bench.ClockSampler(0)
    s.proc = _Done()
    s.lines = [
        "0, 2032, 2032, 812.4, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2032, 1099.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2010, 2032, 1050.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2032, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active",   # skipped
        "truncated, line",                                                                 # skipped
    ]
    out = s.stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2010.0 and out["sm_max_mhz"] == 2032.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_flags_thermal_and_hardware_slowdown(bench):
    s = bench.ClockSampler(0)
    s.proc = _Done()
    s.lines = ["0, 1500, 2032, 700, 0x48, Active, Not Active, Active, Not Active"]
    assert s.stop()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi_says_so(bench):
    out = bench.ClockSampler(0).stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


def test_peaks_come_from_the_measured_file_or_the_stated_fallback(bench, tmp_path, monkeypatch):
    peaks, source = bench._peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert source == "measured" and peaks["hbm_gbs"] > 1000
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, source = bench._peaks()
    assert source == "fallback"
    assert peaks["hbm_gbs"] == 6400.0 and peaks["bf16_tflops"] == 1800.0


def test_fp32_simt_peak_follows_the_unit_count_and_clock(bench):
    assert bench._fp32_simt_peak_tflops(2032.0) == pytest.approx(76.99, abs=0.01)
    assert bench._fp32_simt_peak_tflops(1016.0) == pytest.approx(76.99 / 2, abs=0.01)


def test_kernels_are_classified_by_their_roofline(bench):
    for name in ("sl_inc_defstate", "sl_gather3_scale", "pi_x_tc", "iota_x_tc", "pi_z_fin",
                 "accum_JT", "cube_two_level", "dot_f2", "finalize", "spatial_L", "spec_restrict",
                 "max_norm3", "state_dlam1"):
        assert bench.is_hbm_kernel(name), name
    for name in ("pi_y", "pi_z", "iota_y", "iota_z", "cnn_conv", "cnn_wgrad"):
        assert not bench.is_hbm_kernel(name), name


def test_time_to_residual_takes_the_first_iterate_at_or_below_each_level(bench):
    h1 = [{"t": 0.0, "residual": 1.0}, {"t": 0.5, "residual": 0.08},
          {"t": 1.0, "residual": 0.009}, {"t": 1.5, "residual": 0.004}]
    h2 = [{"t": 0.0, "residual": 1.0}, {"t": 0.7, "residual": 0.1},
          {"t": 1.2, "residual": 0.01}, {"t": 1.9, "residual": 0.0009}]
    out = bench.time_to_residual([h1, h2])
    assert out["0.1"] == pytest.approx((0.5 + 0.7) / 2)
    assert out["0.01"] == pytest.approx((1.0 + 1.2) / 2)
    assert out["0.001"] is None               # h1 never reaches it: no mean over a subset
    assert out["min_residual"] == 0.0009
    assert bench.first_time_at(h2, 1e-3) == 1.9


def test_host_replicas_are_bounded_by_cores_and_memory(bench):
    P, ncpu = bench._host_replicas()
    assert 1 <= P <= ncpu


def test_batched_form_in_the_line_reports_a_failure_instead_of_raising(bench, monkeypatch):
    def broken(args):
        assert args.pairs == bench.BATCH_PAIRS_IN_LINE   # the reduced pair count is passed on
        raise RuntimeError("no device")
    monkeypatch.setattr(bench, "run_batch", broken)
    import argparse
    out = bench.measure_batched_form(argparse.Namespace(pairs=64, batch_threads=16))
    assert out == {"error": "RuntimeError: no device"}


def test_batched_form_keeps_the_throughput_fields(bench, monkeypatch):
    full = {"value": 14.0, "unit": "pairs/s", "config": {"pairs": 16}, "sequential_pairs_per_s": 9.0,
            "speedup_vs_sequential": 1.5, "metric": "dropped", "ms_per_step": 1.0}
    monkeypatch.setattr(bench, "run_batch", lambda args: full)
    import argparse
    out = bench.measure_batched_form(argparse.Namespace(pairs=64, batch_threads=16))
    assert out == {k: full[k] for k in ("value", "unit", "config", "sequential_pairs_per_s",
                                        "speedup_vs_sequential")}
    assert "16 seeded" in bench.batch_workload(16) and "seeds 100-115" in bench.batch_workload(16)
