"""The roofline arithmetic bench.py reports, on made-up counters (no GPU):
achieved = 4 d n flops per seed-iteration x seed-iterations / shift time,
frac = achieved / peak, traffic = the committed DRAM bytes of one
frame-iteration x frame-iterations per launch (null once the kernel source
no longer matches the capture), and the FP32 form's peak from the SM count,
lanes and the sampled clock."""
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

TOT = {"seed_iters": 129793 * 40, "shift_ms": 40 * 3.82, "shift_launches": 40, "frame_iters": 40 * 54.72}
STEPS = [180.0, 181.0]


def _committed(kernel, src):
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    for line in open(bench.TRAFFIC):
        if line.startswith("#") or not line.strip():
            continue
        name, per_unit, src_hash = line.split()[:3]
        if name == kernel:
            return float(per_unit), src_hash == h
    return None, False


def test_tensor_form():
    r = bench.roofline_of("bf16-batched", TOT, STEPS, {"sm_mhz": 2070.0}, 152)
    flops = 4.0 * 16 * 131072 * TOT["seed_iters"]
    assert r["achieved"] == pytest.approx(flops / (TOT["shift_ms"] / 1e3) / 1e12, rel=1e-12)
    peak = bench.load_peaks().get("bf16_tflops_sustained") or 1700.0
    assert r["peak"] == peak and r["frac"] == pytest.approx(r["achieved"] / peak, rel=1e-12)
    assert r["bound"] == "tensor" and r["kernel"] == "k_shift_tc" and r["unit"] == "TFLOP/s"
    assert r["shift_share_of_step"] == pytest.approx(TOT["shift_ms"] / sum(STEPS), rel=1e-12)
    per_unit, current = _committed("k_shift_tc", bench.SHIFT_TC_SRC)
    if current:
        assert r["traffic"] == pytest.approx(per_unit * 54.72, rel=1e-12)
    else:
        assert r["traffic"] is None


def test_fp32_form():
    r = bench.roofline_of("fp32", TOT, STEPS, {"sm_mhz": 2070.0}, 152)
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12, rel=1e-12)   # 80.5 TFLOP/s
    assert r["bound"] == "alu" and r["kernel"] == "k_shift_fp32"
    per_unit, current = _committed("k_shift_fp32", bench.SHIFT_SRC)
    assert (r["traffic"] is not None) == current


def test_no_shift_time_reports_no_rate():
    r = bench.roofline_of("bf16", dict(TOT, shift_ms=0.0), STEPS, {}, 152)
    assert r["achieved"] is None and r["frac"] is None
