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


# ------------------------------------------------------------------ the file
# ZMC_TUNE_CACHE: a first process writes its tuned choices to the file; a
# second process with the same library and GPU takes them from the file
# (edited here, so that taking them shows) and times nothing, skipping lines
# that do not parse or hold values a setter would reject.
CACHE_CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
from paper_1902_07916_gb300 import zmc
out = {}
for name, dim, k, n, trials, prec, tuning in json.loads(sys.argv[2]):
    with zmc.Integrator(dim, [0.0] * dim, [1.0] * dim, k, n, trials, 1, 1.0, 5, "sin_sum", [],
                        precision=zmc.PRECISIONS[prec]) as it:
        zmc.zmc_set_tuning(it.h, tuning)
        r = it.integrate()
        out[name] = [list(zmc.zmc_launch_shape(it.h)), list(r.work_plan)]
print(json.dumps(out))
"""


def cache_child(zmc, path, cases):
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ)
    env.pop("ZMC_TUNE", None)
    env["ZMC_TUNE_CACHE"] = path
    env["ZMC_LIBRARY"] = zmc.LIB_PATH
    r = subprocess.run([sys.executable, "-c", CACHE_CHILD, root, json.dumps(cases)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_tuned_choices_persist_in_the_cache_file(zmc, tmp_path):
    import json
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # a shape-only handle (FP32, d = 4) and a shape + plan handle (FP64,
    # d = 3, level 1 of 2^26 points, inside the plan tuner's 2^31 limit)
    cases = [["shape", 4, 6, 1000, 5, "fp32_fp64acc", zmc.ZMC_TUNE_SHAPE],
             ["plan", 3, 16, 2048, 8, "fp64", zmc.ZMC_TUNE_SHAPE | zmc.ZMC_TUNE_PLAN]]
    path = str(tmp_path / "tune.jsonl")
    first = cache_child(zmc, path, cases)
    lines = [json.loads(x) for x in open(path).read().splitlines()]
    shapes = {(x["kernel"], x["d"]) for x in lines if x["kind"] == "shape"}
    plans = [x for x in lines if x["kind"] == "plan"]
    assert len(lines) == 3 and len(plans) == 1, lines
    assert any(k.startswith("reg/m1/") and d == 4 for k, d in shapes), shapes
    assert any(k.startswith("reg/m0/") and d == 3 for k, d in shapes), shapes
    assert plans[0]["d"] == 3 and plans[0]["n"] == 2048 and plans[0]["tiles"] == 16 ** 3 * 8
    assert plans[0]["plan"] == first["plan"][1]
    for x in lines:
        assert x["device"] == lines[0]["device"] and "/sm%d/" % sms in x["device"]

    # edit the choices: 128 threads and one CTA per SM, another valid plan;
    # add lines the reader must skip
    other_plan = [1 << 17, 256, 64, 1024, 1 << 15]
    edited = []
    for x in lines:
        if x["kind"] == "shape":
            x.update(threads=128, per_sm=1)
            edited.append(json.dumps(dict(x, threads=100)))
        else:
            x["plan"] = other_plan
        edited.append(json.dumps(x))
    edited.insert(0, "not a cache line")
    edited.append('{"kind": "plan", "device": "x", "kernel": "y", "d": 1, "n": 2, '
                  '"tiles": 3, "plan": [0, 0, 0, 0, 0]}')
    text = "\n".join(edited) + "\n"
    with open(path, "w") as fh:
        fh.write(text)
    second = cache_child(zmc, path, cases)
    for name in ("shape", "plan"):
        assert second[name][0] == [128, sms], (name, second[name])
    assert second["plan"][1] == other_plan
    assert second["shape"][1] == DEFAULT_PLAN
    # everything came from the file: nothing was timed, nothing appended
    assert open(path).read() == text
