"""Host logic of bench.py on CPU: the roofline object takes the kernel with the most device
time, divides its algorithmic bytes (or flops) per launch by its average launch time, picks
the roof it is closest to, and scales the measured DRAM/algorithmic ratio into `traffic`."""
import pytest

import bench

PEAK = {"hbm_gbs": 6797.2, "bf16": 1934.6, "source": "measured"}


def _prof(ms, launches, bytes_, flops):
    return {"ms": ms, "launches": launches, "bytes": bytes_, "flops": flops}


def test_dominant_kernel_hbm_roof_and_traffic():
    prof = {
        "local_solve": _prof(100.0, 10, 10 * 16.0e9, 10 * 1.0e9),  # 1.6e10 B per 10 ms launch
        "spmv": _prof(30.0, 10, 10 * 1.0e9, 10 * 1.0e9),
    }
    r = bench.roofline(prof, PEAK, "mixed")
    assert r["kernel"] == "local_solve" and r["bound"] == "hbm"
    assert r["avg_launch_ms"] == pytest.approx(10.0)
    assert r["achieved"] == pytest.approx(16.0e9 / 10e-3 / 1e9)  # 1,600 GB/s
    assert r["frac"] == pytest.approx(1600.0 / 6797.2)
    ratio = bench.DRAM_PER_ALG[("local_solve", "mixed")][0]
    assert r["traffic"] == pytest.approx(ratio * 16.0e9)
    assert r["share_of_device_time"] == pytest.approx(100.0 / 130.0)


def test_alu_roof_and_no_traffic_without_a_capture():
    # 1e12 flop in 10 ms = 100 TFLOP/s against FP32 units; bytes negligible
    prof = {"lu_update": _prof(10.0, 1, 1.0e6, 1.0e12)}
    r = bench.roofline(prof, PEAK, "mixed")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(100.0)
    assert r["peak"] == pytest.approx(bench.FP32_PEAK_TFLOPS)
    assert r["traffic"] is None


def test_rank_seeds_are_distinct():
    assert len({bench.rhs_seed(r) for r in range(8)}) == 8
    assert bench.max_over_ranks(3.5, 1) == 3.5
