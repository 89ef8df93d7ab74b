"""Host-side logic of the benchmark: the closed forms it times accuracy
against, and the median-over-seeds rule of the time-to-accuracy leg."""
import math

import pytest

import bench
from oracle import closed_forms as CF
from paper_1902_07916_gb300 import workloads


@pytest.mark.parametrize("make", [workloads.sin3d, workloads.sin6d, workloads.gauss9d,
                                  lambda: workloads.gauss9d(0.3)])
def test_exact_value_matches_oracle_closed_forms(make):
    w = make()
    assert math.isclose(bench.exact_value(w), CF.integral(w.integrand, w.lo, w.hi, w.params),
                        rel_tol=1e-13, abs_tol=1e-15)


def test_exact_value_textbook_numbers():
    # Im((e^{10i} - 1)/i)^3 and ^6, evaluated independently of either implementation
    z = (complex(math.cos(10.0), math.sin(10.0)) - 1.0) / 1j
    assert math.isclose(bench.exact_value(workloads.sin3d()), (z ** 3).imag, rel_tol=1e-14)
    assert math.isclose(bench.exact_value(workloads.sin6d()), -49.16507381641946, rel_tol=1e-13)
    assert math.isclose(bench.exact_value(workloads.gauss9d()), math.erf(1 / (0.1 * 2 ** 0.5)) ** 9)


def test_median_first():
    assert bench.median_first([4, 2, 8, 1, 16]) == (4, 0)
    assert bench.median_first([None, 2, None, 1, 16]) == (16, 4)
    assert bench.median_first([None, 2, None, 1, None]) == (None, None)
    assert bench.median_first([2, 2, 2, 2, 2]) == (2, 2)


def test_algorithmic_bytes_of_the_benchmark_step():
    # sin6d, FP32 stream: level 1 has 4096 x 10 tiles of ceil(65536 / 11) =
    # 5958 point groups, cut into min(ceil(2^18 / 40960), 5958 // 1024) = 5
    # units each; level 2 has 1,204,224 x 10 tiles, one unit each; 16 bytes
    # per unit, averaged over the two launches
    level1 = 4096 * 10 * 5 * 16
    level2 = 1204224 * 10 * 16
    got = bench.algorithmic_bytes_per_launch([4096, 1204224], 1 << 16, 10, False)
    assert got == (level1 + level2) / 2 == 97976320
    # the FP64 stream: 16384 groups of 4, 7 units per level-1 tile
    got64 = bench.algorithmic_bytes_per_launch([4096], 1 << 16, 10, True)
    assert got64 == 4096 * 10 * 7 * 16


def test_philox_work_per_point():
    # 17 wide multiplies per block; FP64: 1 block per 4 points per dimension,
    # FP32: 2 blocks per 11 points per dimension
    assert bench.philox_multiplies_per_sample(6, True) == 6 * 17 / 4
    assert bench.philox_multiplies_per_sample(6, False) == pytest.approx(6 * 34 / 11, rel=1e-15)


def test_fp32_flop_counts():
    assert bench.fp32_flops_per_sample("sin_sum", 6) == 18
    assert bench.fp32_flops_per_sample("gauss_norm", 9) == 41
    # corner peak: r^(d+1) by binary powering, e = 9 = 0b1001: 4 squarings, 2 products
    assert bench.fp32_flops_per_sample("genz_corner", 8) == 2 * 8 + 4 + 2 + 3


def test_corner_peak_closed_form():
    # the benchmark's exact-rational corner peak against the oracle's, and in
    # 1-D against the antiderivative: int_0^1 (1 + a x)^-2 dx = 1 / (1 + a)
    w = workloads.corner8d()
    assert math.isclose(bench.exact_value(w), CF.integral(w.integrand, w.lo, w.hi, w.params),
                        rel_tol=1e-14)
    assert math.isclose(bench.corner_peak_exact([0.0], [1.0], [3.0]), 0.25, rel_tol=1e-15)
    # 2-D: (1/(2 a b)) [1 - 1/(1+a) - 1/(1+b) + 1/(1+a+b)]
    a, b = 1.5, 4.0
    want = (1 - 1 / (1 + a) - 1 / (1 + b) + 1 / (1 + a + b)) / (2 * a * b)
    assert math.isclose(bench.corner_peak_exact([0.0, 0.0], [1.0, 1.0], [a, b]), want,
                        rel_tol=1e-14)
