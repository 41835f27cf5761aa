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
    assert r["frac_of_nominal"] == pytest.approx(1600.0 / bench.HBM_NOMINAL_GBS)


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


def test_kernel_table_rates_per_step():
    prof = {
        "spmv": _prof(20.0, 10, 10 * 2.0e9, 10 * 1.0e8),   # 2e10 B in 20 ms: 1,000 GB/s
        "local_solve": _prof(60.0, 10, 10 * 30.0e9, 0.0),  # 3e11 B in 60 ms: 5,000 GB/s
        "idle": _prof(0.0, 0, 0.0, 0.0),
    }
    t = bench.kernel_table(prof, PEAK, steps=5)
    assert list(t) == ["local_solve", "spmv"]  # by device time, launched kernels only
    s = t["spmv"]
    assert s["ms_per_step"] == pytest.approx(4.0) and s["launches_per_step"] == 2
    assert s["bytes_per_launch"] == pytest.approx(2.0e9) and s["flops_per_launch"] == pytest.approx(1.0e8)
    assert s["gbs"] == pytest.approx(1000.0) and s["tflops"] == pytest.approx(1.0e9 / 0.02 / 1e12)
    assert s["hbm_frac"] == pytest.approx(1000.0 / 6797.2)
    assert t["local_solve"]["hbm_frac_of_nominal"] == pytest.approx(5000.0 / bench.HBM_NOMINAL_GBS)


def test_oracle_baselines_on_a_tiny_workload():
    """The single-thread sample (one-thread spawned worker) and the pool-against-pool all-core
    estimate run end to end: 10^3 cells, 2^3 subdomains, every box shape sampled."""
    W = dict(bench.WORKLOADS["maxwell60_k30_2lvl"], n=10, coarse=0, nrhs=2)
    s = bench.cpu_baseline(W, 10, budget_s=2.0)
    assert s["cores"] == 1 and s["value"] > 0 and s["t_fac"] > 0 and s["t_fac_largest"] >= s["t_fac"] * 0.5
    assert "8 subdomains" in s["sample"]
    a = bench.cpu_baseline_allcore(W, 10, s, budget_s=1.0)
    assert a["cores"] >= 1 and a["value"] > 0
    assert "1-process pool" in a["sample"]
