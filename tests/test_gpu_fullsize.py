"""Parity at the full workload sizes, in the launch configuration the
benchmark times.

The oracle cannot run a 10^11-point tree, but the stream is counter-based, so
any (cell, trial) of any level can be recomputed on its own: sampled tiles of
every level are recomputed by the oracle and compared with the kernel's sums;
every level's threshold and flags are re-derived from the kernel's own
per-cell spreads; the final value is re-summed from the accepted cells.
"""
import math

import numpy as np
import pytest

from oracle import zmc_oracle as O
from paper_1902_07916_gb300 import workloads

from parity import check_decisions_consistent, level_coords, run_gpu, sums_tolerance

pytestmark = pytest.mark.gpu

SAMPLED_TILES = 24


@pytest.fixture(scope="module")
def zmc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_07916_gb300 import build
    build.build()
    from paper_1902_07916_gb300 import zmc as mod
    return mod


def sampled_parity(w, levels, fp32, rtol):
    rng = np.random.default_rng(1234)
    coords = level_coords(w, levels)
    for L, g in enumerate(levels, start=1):
        if g["cells"] == 0:
            break
        C = g["cells"]
        cells = np.unique(np.concatenate([[0, C - 1], rng.integers(0, C, SAMPLED_TILES)]))
        ref = O.cell_sums(w.seed, L, w.lo, w.hi, w.k, w.n, w.trials, w.integrand, w.params,
                          cells, coords[L - 1][cells], fp32_uniforms=fp32)
        got = g["sums"][cells]
        err = np.abs(got - ref)
        tol = sums_tolerance(ref, w.n, rtol)
        if fp32:
            # FP32 flushes values below ~1e-38 (a Gaussian tail, its squares):
            # an absolute floor 12 orders below the level's largest tile.
            all_sums = g["sums"]
            level_scale = float(np.max(np.abs(all_sums[..., 0])
                                       + np.sqrt(w.n * np.abs(all_sums[..., 1]))))
            tol = tol + 1e-12 * level_scale
        assert np.all(err <= tol), (L, float(err.max()))


def test_bench_workload_fp32_full_size(zmc):
    # the benchmark's step: sin(sum x), 6-D, k=4, n=2^16, 10 trials, depth 3,
    # m=1.5, default budget, FP32 evaluation with FP64 accumulation
    w = workloads.sin6d()
    res, levels = run_gpu(zmc, w, "fp32_fp64acc")
    assert res.levels_run >= 2 and res.flagged_per_level[0] > 0
    sampled_parity(w, levels, fp32=True, rtol=2e-5)
    check_decisions_consistent(w, levels, res)


def test_corner_peak_fp64_full_size(zmc):
    w = workloads.corner8d()
    res, levels = run_gpu(zmc, w, "fp64")
    sampled_parity(w, levels, fp32=False, rtol=1e-12)
    check_decisions_consistent(w, levels, res)


def test_gaussian_9d_fp32_full_size(zmc):
    w = workloads.gauss9d()
    res, levels = run_gpu(zmc, w, "fp32_kahan")
    sampled_parity(w, levels, fp32=True, rtol=2e-5)
    check_decisions_consistent(w, levels, res)
    # the closed form is 1 to double precision
    assert abs(res.value - 1.0) <= 4 * res.std
