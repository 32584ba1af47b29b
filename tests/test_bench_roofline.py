"""bench.py's roofline arithmetic on CPU: the bound chosen for the level-0 A
product, the achieved figure over the measured peak, and the DRAM traffic
estimate, checked against the per-launch figures of a recorded run of the
616k-node tube (224.6 us FP64 launches of 782.9 MB and 2 flops per stored
scalar; 110.4 us FP32 launches of 410.8 MB)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
bench = pytest.importorskip("bench")

HBM = 6781.4           # GB/s, the measured copy bandwidth the bench divides by
CLOCKS = {"sm_mhz": 2070.0}
BLOCKS = 9_040_000     # stored 3x3 blocks of A on the 616k-node tube
LAUNCHES = 2527


def _kprof(us_per_launch, bytes_per_launch, flops_per_launch, timed=LAUNCHES):
    return {"launches": LAUNCHES, "timed": timed, "ms": us_per_launch * timed * 1e-3,
            "bytes": bytes_per_launch * timed, "flops": flops_per_launch * timed}


def test_fp64_product_is_bound_by_the_fp64_pipe():
    flops = 2.0 * 9 * BLOCKS
    r = bench.roofline(_kprof(224.6, 782.86e6, flops), True, CLOCKS, 1070.0, HBM, "measured",
                       "level-0 A product (FP64 values)", 102)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    # 2 FMA per SM per clock, 152 SMs, 2.07 GHz, 2 flops per FMA
    assert r["peak"] == pytest.approx(2 * 2 * 152 * 2.07e9 * 1e-12)
    assert r["achieved"] == pytest.approx(flops / 224.6e-6 * 1e-12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["frac"] == pytest.approx(0.576, abs=2e-3)
    assert r["hbm_frac"] == pytest.approx(782.86e6 / 224.6e-6 / (HBM * 1e9))
    assert r["hbm_frac"] == pytest.approx(0.514, abs=2e-3)
    assert r["share_of_step"] == pytest.approx(224.6 * LAUNCHES * 1e-3 / 1070.0)
    # the captured scalar-row kernel: DRAM traffic = ncu ratio x algorithmic bytes
    assert r["traffic"] == pytest.approx(bench.TRAFFIC_RATIO["fp64"] * 782.86e6)


def test_fp32_product_is_bound_by_hbm():
    r = bench.roofline(_kprof(110.4, 410.75e6, 2.0 * 9 * BLOCKS), False, CLOCKS, 617.5, HBM, "measured",
                       "level-0 A product (FP32 values)", 102)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == HBM
    assert r["achieved"] == pytest.approx(410.75e6 / 110.4e-6 * 1e-9)
    assert r["frac"] == pytest.approx(0.549, abs=2e-3)
    assert r["traffic"] == pytest.approx(bench.TRAFFIC_RATIO["fp32"] * 410.75e6)


def test_traffic_is_null_without_a_capture_of_the_kernel():
    kp = _kprof(101.4, 410.75e6, 2.0 * 9 * BLOCKS)
    # the 16-byte kernel (code 304) has no DRAM capture in its current form
    assert bench.roofline(kp, False, CLOCKS, 592.5, HBM, "measured", "A", 304)["traffic"] is None
    assert bench.roofline(kp, False, CLOCKS, 592.5, HBM, "measured", "A", 102, captured=False)["traffic"] is None
    assert bench.roofline(kp, False, CLOCKS, 592.5, HBM, "measured", "A", 304)["frac"] == pytest.approx(
        0.597, abs=2e-3)


def test_no_profile_gives_no_roofline():
    assert bench.roofline(None, True, CLOCKS, 1.0, HBM, "measured", "A", 102) is None
    assert bench.roofline(_kprof(1.0, 1.0, 1.0, timed=0), True, CLOCKS, 1.0, HBM, "measured", "A", 102) is None


def test_traffic_ratios_are_the_captured_ones():
    # dram read + write over algorithmic bytes of the captured Chebyshev-step launches
    assert bench.TRAFFIC_RATIO["fp64"] == pytest.approx(396.7 / 403.6)
    assert bench.TRAFFIC_RATIO["fp32"] == pytest.approx(206.5 / 211.4)
