"""bench.py's measurement bookkeeping, on the CPU: the summary of nvidia-smi samples taken
during a timed region (median SM clock under load, maximum clock, throttle reasons) and
the source of the HBM peak (the measured file, else the stated fallback)."""
import importlib.util
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def bench_module():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(os.path.dirname(HERE), "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def summary_of(lines):
    sampler = bench_module().ClockSampler(0)
    sampler.out = "\n".join(lines)
    return sampler.summary()


def test_median_under_load_and_no_reasons():
    rows = ["0, 2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active"] * 5
    rows += ["0, 345, 2070, 120.0, Not Active, Not Active, Not Active, Not Active"]  # idle sample
    s = summary_of(rows)
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["reasons"] == [] and s["samples"] == 6


def test_throttle_reasons_are_reported():
    rows = ["0, 1800, 2070, 1400.0, Not Active, Not Active, Not Active, Active",
            "0, 1750, 2070, 1400.0, Not Active, Active, Not Active, Active",
            "0, 1790, 2070, 1400.0, Not Active, Not Active, Not Active, Not Active"]
    s = summary_of(rows)
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert s["sm_mhz"] == 1790.0


def test_unsampled_when_nvidia_smi_gave_nothing():
    s = summary_of(["", "garbage line"])
    assert s["sm_mhz"] is None and s["reasons"] == ["unsampled"]


def test_hbm_peak_from_the_measured_file_else_the_fallback(tmp_path):
    b = bench_module()
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6774.6, "bf16_tflops": 1900}')
    assert b._hbm_peak(str(tmp_path)) == (6774.6, "MEASURED_PEAKS.json hbm_gbs (of measured)")
    empty = tmp_path / "none"
    empty.mkdir()
    peak, source = b._hbm_peak(str(empty))
    assert peak == 6800.0 and "fallback" in source
