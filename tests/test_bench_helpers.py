"""CPU checks of the benchmark's host-side arithmetic: the per-class DRAM
traffic of the mean product launch, the peak each precision is measured
against, and the `config` every precision choice reports."""

import pytest

import bench


def test_mean_launch_traffic_separates_the_product_classes():
    # a solve with f32 FP64-equivalent flops of FP32-class products (10 slice
    # products each) and f64 of FP64-class ones (28 each)
    f32, f64, launches = 3.0e12, 1.0e12, 50
    tensor = 10.0 * f32 + 28.0 * f64
    want = (f32 * bench.TRAFFIC_PER_FLOP["fp32"] + f64 * bench.TRAFFIC_PER_FLOP["fp64_tc"]) / launches
    for prec in ("fp32", "fp32_refine"):
        assert bench.mean_launch_traffic(prec, f32 + f64, tensor, launches) == pytest.approx(want, rel=1e-12)
    # every product FP64 class
    got = bench.mean_launch_traffic("fp64_tc", f64, 28.0 * f64, launches)
    assert got == pytest.approx(f64 * bench.TRAFFIC_PER_FLOP["fp64_tc"] / launches, rel=1e-12)
    # classes without a captured figure, or no launches
    assert bench.mean_launch_traffic("fp64", f64, 0.0, launches) is None
    assert bench.mean_launch_traffic("mixed_bf16", f64, 0.0, launches) is None
    assert bench.mean_launch_traffic("fp32", f64, 10.0 * f64, 0) is None


def test_traffic_per_flop_is_that_of_one_captured_launch():
    # the captured 3072 x 3072 x 4096 launches read and wrote about 1 GB
    # (FP32 class) and 3.3 GB (FP64 class)
    ref = bench.TRAFFIC_REF_FLOPS
    assert 0.9e9 < bench.TRAFFIC_PER_FLOP["fp32"] * ref < 1.2e9
    assert 3.0e9 < bench.TRAFFIC_PER_FLOP["fp64_tc"] * ref < 3.6e9


def test_dominant_peak_per_precision():
    peaks = {"hbm_gbs": 6790.3, "bf16_tflops": 1872.0, "bf16_tflops_sustained": 1693.5}
    p64, note = bench.dominant_peak("fp64", peaks)
    assert p64 == pytest.approx(1693.5 * 1.25 / 2250.0) and "nominal" in note
    for prec in ("fp32_refine", "fp32", "fp64_tc", "mixed_bf16"):
        p, _ = bench.dominant_peak(prec, peaks)
        assert p == 1693.5


@pytest.mark.parametrize("prec", ["fp32_refine", "fp32", "fp64_tc", "fp64", "mixed_bf16"])
def test_every_precision_choice_has_a_config(prec):
    c = bench.bench_config(prec, 1)
    assert c["workload"] == bench.WORKLOAD and c["prec"] == prec and c["schedule"]
    assert c["parallelism"] == "replicas1"
