"""The autotuner and the work plan (zmc_set_tuning, zmc_set_work_plan).

The launch shape never changes a result (test_gpu_batch_expr checks four
shapes bit for bit).  The work plan -- how a level is cut into units, i.e.
samples per thread and when a whole tile runs on one lane -- decides the
order of summation, so every result records it: here a non-default plan
still matches the oracle to the FP64 tolerance, a tuned plan reproduces bit
for bit when passed back through zmc_set_work_plan, and tuning is not slower
than the default on two workloads where the plan's rules matter."""
import time

import pytest

from paper_1902_07916_gb300.workloads import Workload

from parity import compare_fp64, run_oracle

pytestmark = pytest.mark.gpu

DEFAULT_PLAN = [1 << 18, 1024, 64, 1024, 1 << 18]


@pytest.fixture(scope="module")
def zmc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_07916_gb300 import build
    build.build()
    from paper_1902_07916_gb300 import zmc as mod
    return mod


def integrator(zmc, w, precision, plan=None, tuning=None):
    it = zmc.Integrator(w.dim, w.lo, w.hi, w.k, w.n, w.trials, w.depth, w.sigma_multiplier,
                        w.seed, w.integrand, w.params, precision=zmc.PRECISIONS[precision])
    if tuning is not None:
        zmc.zmc_set_tuning(it.h, tuning)
    if plan is not None:
        zmc.zmc_set_work_plan(it.h, plan)
    return it


def test_results_record_the_default_plan(zmc):
    w = Workload("sin3", "sin_sum", 3, [0.0] * 3, [10.0] * 3, 4, 1000, 5, 2, 2.0, 0)
    with integrator(zmc, w, "fp64") as it:
        assert it.integrate().work_plan == DEFAULT_PLAN


def test_other_plan_still_matches_the_oracle(zmc):
    # lane tiles on a 40,960-tile level and 256-group units elsewhere: another
    # order of summation, the same sums to the FP64 tolerance, same decisions
    w = Workload("sin6_tiles", "sin_sum", 6, [0.0] * 6, [10.0] * 6, 4, 256, 10, 2, 1.5, 2)
    plan = [1 << 17, 256, 64, 1024, 1 << 15]
    it = integrator(zmc, w, "fp64", plan=plan)
    try:
        it.trace(True)
        res = it.integrate()
        levels = [it.trace_level(L) for L in range(1, w.depth + 1)]
    finally:
        it.close()
    assert res.work_plan == plan
    compare_fp64(w, res, levels, run_oracle(w))


def best_of(it, runs=3):
    it.integrate()
    ts = []
    for _ in range(runs):
        t0 = time.perf_counter()
        r = it.integrate()
        ts.append(time.perf_counter() - t0)
    return min(ts), r


TUNE_CASES = [
    # moderate tiles (256 point groups) on a level of 125,000 tiles
    Workload("sin6_k5", "sin_sum", 6, [0.0] * 6, [10.0] * 6, 5, 1280, 8, 1, 1.0, 3),
    # small tiles of a 9-D Gaussian (64 groups) on a level of 157,464 tiles
    Workload("gauss9_n320", "genz_gauss", 9, [0.0] * 9, [1.0] * 9, 3, 320, 8, 1, 1.0, 4,
             [2.0] * 9 + [0.5] * 9),
]


@pytest.mark.parametrize("w", TUNE_CASES, ids=[w.name for w in TUNE_CASES])
def test_tuned_plan_is_not_slower_and_reproduces(zmc, w):
    with integrator(zmc, w, "fp32_fp64acc") as base:
        t_default, r_default = best_of(base)
    with integrator(zmc, w, "fp32_fp64acc",
                    tuning=zmc.ZMC_TUNE_SHAPE | zmc.ZMC_TUNE_PLAN) as tuned:
        t_tuned, r_tuned = best_of(tuned)
    assert r_default.work_plan == DEFAULT_PLAN
    assert t_tuned <= 1.10 * t_default, (t_tuned, t_default, r_tuned.work_plan)
    # the recorded plan, set explicitly on a fresh handle, gives the same bits
    with integrator(zmc, w, "fp32_fp64acc", plan=r_tuned.work_plan) as again:
        r = again.integrate()
    assert (r.value, r.std, r.flagged_per_level) == (r_tuned.value, r_tuned.std,
                                                     r_tuned.flagged_per_level)
    assert r.work_plan == r_tuned.work_plan
