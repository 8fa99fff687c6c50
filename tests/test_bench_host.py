"""Host-side logic of bench.py that needs no GPU: the clock record's parsing of nvidia-smi
samples (median SM clock, maximum clock, throttle reasons), the GPU selector, the measured
peaks and their fallback, the guard that drops the committed ncu traffic figure once the
kernel source changes, and the reference arm's JSON line (the oracle on the host cores)."""
import json
import os
import shutil
import types

import pytest

import bench


class _FakeProc:
    def __init__(self, out):
        self.out = out

    def terminate(self):
        pass

    def kill(self):
        pass

    def communicate(self, timeout=None):
        return self.out, ""


def _sampler(out):
    c = bench.ClockSampler.__new__(bench.ClockSampler)
    c.dev, c.gpu, c.p = 0, "GPU-test", _FakeProc(out)
    return c


def test_clock_record_median_max_and_reasons():
    # index, sm, max sm, power, active, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    out = "\n".join([
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2055, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    r = _sampler(out).stop()
    assert r["sm_mhz"] == 2055 and r["sm_max_mhz"] == 2070
    assert r["reasons"] == ["sw_power_cap"] and r["samples"] == 3 and r["gpu"] == "GPU-test"


def test_clock_record_lists_every_slowdown_reason_once():
    out = "\n".join([
        "0, 1500, 2070, 1000, 0x8, Active, Not Active, Active, Not Active",
        "0, 1400, 2070, 1000, 0x8, Active, Active, Not Active, Not Active",
    ])
    r = _sampler(out).stop()
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert r["sm_mhz"] == 1450


def test_clock_record_without_nvidia_smi():
    c = bench.ClockSampler.__new__(bench.ClockSampler)
    c.p = None
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_gpu_selector_maps_the_ordinal_through_visible_devices(monkeypatch):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("the UUID path is taken on a GPU machine")
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "GPU-aaaa, GPU-bbbb")
    assert bench.gpu_id(1) == "GPU-bbbb"
    monkeypatch.delenv("CUDA_VISIBLE_DEVICES")
    assert bench.gpu_id(0) == "0"


def test_peaks_measured_and_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks()[3] == "fallback"
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps(
        {"hbm_gbs": 6781.1, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1715.0, "sm_max_mhz": 2070}))
    hbm, bf16, mhz, src = bench.peaks()
    # kernels timed inside a long step take the sustained bf16 figure
    assert (hbm, bf16, mhz, src) == (6781.1, 1715.0, 2070, "measured")


def test_traffic_figure_dropped_once_the_kernel_source_changes(tmp_path, monkeypatch):
    root = os.path.dirname(os.path.abspath(bench.__file__))
    with open(os.path.join(root, "profiles", "ncu_traffic.json")) as fh:
        rec = json.load(fh)["xline"]
    # the committed record matches the committed source
    assert bench.kernel_traffic("xline") == rec["bytes_per_launch_scaled"]
    assert bench.kernel_traffic("no_such_class") is None
    # a copy of the tree whose kernel source differs by one byte
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(root, "profiles", "ncu_traffic.json"), tmp_path / "profiles")
    src_dir = tmp_path / "paper_2604_11139_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    src = os.path.join(root, "paper_2604_11139_gb300", "csrc", rec["source"])
    shutil.copy(src, src_dir)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("xline") == rec["bytes_per_launch_scaled"]
    with open(src_dir / rec["source"], "ab") as fh:
        fh.write(b"\n")
    assert bench.kernel_traffic("xline") is None


def test_weak_value_sums_the_replicas():
    assert bench.weak_value(1, 600, 2.0) == pytest.approx(300.0)
    assert bench.weak_value(4, 600, 2.0) == pytest.approx(1200.0)


def test_reference_arm_line(capsys, monkeypatch):
    monkeypatch.delenv("RANK", raising=False)
    args = types.SimpleNamespace(workload="tiny_gamma_fp64", steps=2, warmup=1, gpus=1)
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["steps"] == 2 and line["warmup"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["higher_is_better"] is True and line["config"]["workload"].startswith("tiny_gamma_fp64")


def test_reference_arm_other_ranks_do_no_work(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    args = types.SimpleNamespace(workload="tiny_gamma_fp64", steps=2, warmup=1, gpus=2)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
