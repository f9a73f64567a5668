"""Host logic of bench.py that needs no GPU: argument defaults, the roofline
assembled from a step's aggregates, and the clock sampler (with a stand-in
nvidia-smi that prints fixed samples)."""
import math
import os
import stat
import sys
import time
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def aggregates():
    # the shape of three default steps (64 blocks each, n = 4096, k = 8)
    return {"gemm_flops": 2.58e13, "inv_flops": 7.6e12, "gemm_device_seconds": 0.73, "inv_device_seconds": 1.37,
            "launches": 2316, "gemm_launches": 42, "inversions": 28416, "peak_device_bytes": 1 << 36,
            "pack_device_seconds": 0.17, "inv_panel_device_seconds": 0.644, "inv_panel_flops": 5.4e11,
            "inv_update_flops": 7.1e12, "inv_panel_launches": 216}


def test_parse_defaults(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert (a.gpus, a.precision, a.n, a.k, a.blocks_per_step, a.together) == (1, "fp64_tc", 4096, 8, 64, 64)
    assert a.refine == 1 and a.warmup >= 3
    monkeypatch.setattr(sys, "argv", ["bench.py", "--precision", "mixed"])
    assert bench.parse().refine == 0


@pytest.mark.parametrize("precision", ["fp64_tc", "fp64", "fp32", "mixed"])
def test_roofline_fields(precision):
    args = types.SimpleNamespace(precision=precision, slices=3)
    r = bench.roofline_of(args, aggregates(), 2.33)
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic", "kernel", "families"):
        assert key in r, key
    assert r["bound"] in ("tensor", "alu") and r["unit"] == "TFLOP/s"
    assert math.isclose(r["frac"], r["achieved"] / r["peak"])
    # the head is the family with the most device time
    fams = {k: v for k, v in r["families"].items() if "bound" in v}
    assert r["kernel"] == max(fams, key=lambda k: fams[k]["device_seconds"])
    if precision == "fp64_tc":
        tr = r["families"]["gj_trailing_update"]
        assert tr["traffic"] == pytest.approx(bench.UPDATE_DRAM_BYTES_PER_FLOP * 7.1e12 / 216)
        assert r["families"]["gj_panel_kernel"]["traffic"] == pytest.approx(
            bench.PANEL_DRAM_BYTES_PER_FLOP * 5.4e11 / 216)
        assert r["families"]["oz_gemm_kernel"]["traffic"] == pytest.approx(
            bench.SCHUR_DRAM_BYTES_PER_FLOP * 2.58e13 / 42)
        # executed digit-pair flops, 36 per FP64 product
        assert r["families"]["oz_gemm_kernel"]["achieved"] == pytest.approx(2.58e13 * 36 / 0.73 / 1e12)
    else:
        assert r["traffic"] is None


def test_clock_sampler_summary(tmp_path, monkeypatch):
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/bash\nwhile true; do\n"
                    "echo '0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Active'\n"
                    "sleep 0.05; done\n")
    fake.chmod(fake.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    c = bench.Clocks(0)
    c.start()
    time.sleep(0.5)
    r = c.stop()
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["reasons"] == ["sw_power_cap"]
    assert r["samples"] >= 2
    assert not os.path.exists(c.path)  # the samples file is removed


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    c = bench.Clocks(0)
    c.start()
    r = c.stop()
    assert r["sm_mhz"] is None and r["reasons"] == ["nvidia-smi unavailable"]


def test_reference_arm_line():
    """`bench.py --impl reference` times the oracle on the host and prints one
    JSON line with the same metric and unit, marked as the reference."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "256", "--k",
                          "4", "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=300,
                         cwd=ROOT, check=True).stdout
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "blocks/s"
    assert d["higher_is_better"] is True and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "blocks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_single_thread():
    """`--cpu-threads 1` runs the oracle on one host thread and says so."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "256", "--k",
                          "4", "--steps", "1", "--warmup", "0", "--cpu-threads", "1"], capture_output=True, text=True,
                         timeout=300, cwd=ROOT, check=True).stdout
    d = json.loads([l for l in out.splitlines() if l.startswith("{")][0])
    assert d["cpu_baseline"]["cores"] == 1 and d["value"] > 0
