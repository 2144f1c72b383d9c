"""Host-side pieces of bench.py that need no GPU: the nvidia-smi clock
samples are kept only inside the timed window (by their timestamps), and
throttle reasons seen there are reported."""
import time

import bench


def _line(t, mhz, power_cap=False):
    stamp = time.strftime("%Y/%m/%d %H:%M:%S", time.localtime(t)) + ".%03d" % int(1000 * (t % 1.0))
    cap = "Active" if power_cap else "Not Active"
    return f"{stamp}, 0, {mhz}, 2070, 900.00, 0x0, Not Active, Not Active, Not Active, {cap}"


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        pass


def _clocks(tmp_path, t0, lines):
    c = bench._Clocks.__new__(bench._Clocks)
    c.path = str(tmp_path / "clocks.csv")
    (tmp_path / "clocks.csv").write_text("\n".join(lines) + "\n")
    c.p = _Proc()
    c.f = open(str(tmp_path / "unused"), "w")
    c.t0 = t0
    c.spans = {}
    c.windows = {}
    return c


def test_timestamp_parse():
    t = 1_800_000_000.25
    s = time.strftime("%Y/%m/%d %H:%M:%S", time.localtime(t)) + ".250"
    assert abs(bench._Clocks._stamp(s) - t) < 1e-6
    assert bench._Clocks._stamp("not a time") is None


def test_window_keeps_samples_inside(tmp_path, monkeypatch):
    now = time.time()
    t0 = now - 1.0
    lines = [_line(t0 - 2.0, 1000), _line(t0 + 0.2, 2070), _line(t0 + 0.5, 2070, power_cap=True),
             _line(t0 + 0.8, 2040), _line(now + 3.0, 500)]
    c = _clocks(tmp_path, t0, lines)
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    r = c.stop()
    assert r["samples"] == 3 and r["sm_mhz"] == 2070.0 and r["reasons"] == ["sw_power_cap"]


def test_short_window_takes_the_neighbouring_samples(tmp_path, monkeypatch):
    now = time.time()
    t0 = now - 0.01                      # shorter than the sampling interval
    lines = [_line(t0 - 0.5, 2000), _line(now + 0.5, 2070)]
    c = _clocks(tmp_path, t0, lines)
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    r = c.stop()
    assert r["samples"] == 2 and r["sm_mhz"] == 2035.0


def test_tensor_roofline_fraction(tmp_path, monkeypatch):
    r = bench._tensor_roofline(288.0)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert abs(r["frac"] - 288.0 / r["peak"]) < 1e-12
    # without the measured peaks the fallback figure is used and said so
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    r = bench._tensor_roofline(190.0)
    assert r["peak"] == 1900.0 and r["peak_source"].startswith("fallback") and abs(r["frac"] - 0.1) < 1e-12


def test_reference_arm_json_line():
    """`bench.py --impl reference` (the FP64 oracle on the host cores) prints
    one JSON line with the GPU arm's metric and unit, the impl marker, its
    CPU baseline and an end-to-end entry without device copies."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]


def test_window_of_a_named_span(tmp_path, monkeypatch):
    now = time.time()
    t0 = now - 1.0
    lines = [_line(t0 - 3.0, 1500), _line(t0 - 2.5, 1600), _line(t0 + 0.5, 2070)]
    c = _clocks(tmp_path, t0, lines)
    c.spans["probe"] = [t0 - 3.1, t0 - 2.4]
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    r = c.stop()
    assert r["samples"] == 1 and r["sm_mhz"] == 2070.0
    assert c.windows["probe"]["samples"] == 2 and c.windows["probe"]["sm_mhz"] == 1550.0


def test_alu_roofline_uses_the_method_costs():
    """frac = (tests x 20 + far x 12 + triangles x 160) flops / time / FP32
    peak, the MUFU co-bound (far x 3 + triangles x 3) beside it; the larger
    fraction names the binding pipe."""
    peaks = {"fp32_tflops": 80.0, "mufu_gops": 5000.0}
    w = {"test": 1000, "far": 500, "leaf": 40}
    r = bench._alu_roofline(w, 1e-3, peaks, "tri")        # 1 us
    flops = 1000 * 20 + 500 * 12 + 40 * 160
    mufu = 500 * 3 + 40 * 3
    assert r["work_per_launch"]["flops"] == flops and r["work_per_launch"]["mufu_ops"] == mufu
    f32 = flops / 1e-6 / 1e12 / 80.0
    fmu = mufu / 1e-6 / 1e9 / 5000.0
    assert r["binding_pipe"] == ("fp32" if f32 >= fmu else "mufu")
    assert abs(r["frac"] - max(f32, fmu)) < 1e-12 and abs(r["co_bound"]["frac"] - min(f32, fmu)) < 1e-12
    # a MUFU-heavy unit mix binds on the MUFU pipe
    r = bench._alu_roofline({"test": 0, "far": 1000, "leaf": 0}, 1e-3, {"fp32_tflops": 80.0, "mufu_gops": 100.0})
    assert r["binding_pipe"] == "mufu" and r["unit"] == "Gop/s"
    assert abs(r["frac"] - 3000 / 1e-6 / 1e9 / 100.0) < 1e-12


def test_peaks_scale_with_the_clock():
    p = {"fp32_tflops": 80.0, "mufu_gops": 5000.0}
    s = bench._scale_peaks(p, 2000.0, 1500.0)
    assert abs(s["fp32_tflops"] - 60.0) < 1e-12 and abs(s["mufu_gops"] - 3750.0) < 1e-9
    assert bench._scale_peaks(p, None, 1500.0)["fp32_tflops"] == 80.0
