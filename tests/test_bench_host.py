"""Host logic of bench.py's roofline object (no GPU): the peak a tensor-core kernel is measured against
follows the timed region (burst under a second without the power cap, sustained otherwise), and the
achieved rate is the algorithmic work per launch over the mean launch time."""
import importlib.util
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(HERE, "..", "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


PEAKS = {"hbm_gbs": 6692.8, "bf16_tflops": 1889.9, "bf16_tflops_sustained": 1730.1}


def _dom(name, launches, ms, flops=0.0, nbytes=0.0):
    return {"name": name, "launches": launches, "ms": ms, "flops": flops, "bytes": nbytes}


def test_tensor_kernel_short_region_uses_burst_peak(bench):
    # 10 launches of 1.8e12 flop in 10 ms: 1800 TFLOP/s
    r = bench.roofline_of(_dom("tc_gemm.crt", 10, 10.0, flops=1.8e13), 100.0, [], PEAKS, "measured")
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(1800.0)
    assert r["peak"] == PEAKS["bf16_tflops"]
    assert r["frac"] == pytest.approx(1800.0 / 1889.9, abs=1e-4)
    assert "burst" in r["peak_source"] and "no power cap" in r["peak_source"]


@pytest.mark.parametrize("total_ms,reasons", [(1500.0, []), (100.0, ["sw_power_cap"])])
def test_tensor_kernel_long_or_capped_region_uses_sustained_peak(bench, total_ms, reasons):
    r = bench.roofline_of(_dom("tc_gemm.crt", 4, 8.0, flops=1.2e13), total_ms, reasons, PEAKS, "measured")
    assert r["peak"] == PEAKS["bf16_tflops_sustained"]
    assert r["achieved"] == pytest.approx(1500.0)
    assert "sustained" in r["peak_source"]


def test_memory_bound_kernel_uses_copy_bandwidth(bench):
    # 2 launches of 6.7 GB in 2 ms: 6700 GB/s
    r = bench.roofline_of(_dom("oz_residues", 2, 2.0, nbytes=1.34e10), 100.0, [], PEAKS, "measured")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(6700.0)
    assert r["peak"] == PEAKS["hbm_gbs"]
    assert r["traffic"] is None


def test_fallback_peaks_when_the_measured_file_lacks_a_key(bench):
    r = bench.roofline_of(_dom("tc_gemm.crt", 1, 1.0, flops=1.0e12), 10.0, [], {}, "fallback")
    assert r["peak"] == 1889.9 and r["peak_source"].startswith("fallback")
