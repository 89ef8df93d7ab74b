"""GPU tests of the batched form (zmc_integrate_batch) and of expression
integrands compiled at run time.

Batch: every integral's result equals its single-integral result bit for
bit (same sampling units, same selection grid), in all three precision
modes, and FP64 batch results match the oracle.  Expressions: an expression
for a registry integrand reproduces it to rounding; expressions with
parameters, conditionals, logic and special functions match the oracle's
expression evaluator element by element (FP64: 1e-12 with identical
decisions; FP32 modes: the FP32 tolerance on every level) and their closed
forms within 3 standard deviations; a bad expression reports
ZMC_ERR_COMPILE with the compiler's log.
"""
import math

import numpy as np
import pytest

from oracle import closed_forms as CF
from paper_1902_07916_gb300.workloads import Workload, genz_batch

from parity import (check_decisions_consistent, compare_fp64,
                    fp32_levels_against_oracle, run_gpu, run_oracle)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zmc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_07916_gb300 import build
    build.build()
    from paper_1902_07916_gb300 import zmc as mod
    return mod


def handles(zmc, ws, precision):
    hs = []
    for w in ws:
        h = zmc.zmc_create(w.dim, w.lo, w.hi, w.k, w.n, w.trials, w.depth, w.sigma_multiplier,
                           w.seed)
        zmc.zmc_set_integrand(h, w.integrand, w.params)
        zmc.zmc_set_precision(h, precision)
        if w.max_cells is not None or w.max_samples is not None:
            zmc.zmc_set_limits(h, w.max_cells or (1 << 24), w.max_samples or (1 << 40))
        hs.append(h)
    return hs


def mixed_batch():
    ws = genz_batch(24, seed=7, trials=4, m=1.0, cap_level1=1 << 22)
    # smaller n for the test, ragged on purpose; a cell budget keeps the
    # deeper levels small enough for the oracle
    ws = [w.with_(n=max(5, w.n // 64 + (i % 4)), max_cells=max(w.k ** w.dim, 4096))
          for i, w in enumerate(ws)]
    W = lambda *a, **k: Workload(*a, **k)
    ws += [
        W("sin3", "sin_sum", 3, [0.0] * 3, [10.0] * 3, 4, 203, 5, 2, 2.0, 0),
        W("gauss3", "gauss_norm", 3, [-1.0] * 3, [1.0] * 3, 3, 77, 4, 3, 1.0, 5, [0.2]),
        W("const2", "constant", 2, [0.0] * 2, [2.0] * 2, 3, 16, 2, 2, 1.0, 1, [3.0]),
        W("lin5", "linear", 5, [0.0] * 5, [1.0] * 5, 2, 41, 3, 2, 0.5, 2,
          [0.5, 1.0, -1.0, 2.0, 0.25, 3.0]),
    ]
    return ws


@pytest.mark.parametrize("precision", ["fp64", "fp32_fp64acc", "fp32_kahan"])
def test_batch_equals_single_runs(zmc, precision):
    ws = mixed_batch()
    hs = handles(zmc, ws, precision)
    try:
        batch = zmc.zmc_integrate_batch(hs)
        again = zmc.zmc_integrate_batch(hs)          # graph replay
        for w, h, b, b2 in zip(ws, hs, batch, again):
            s = zmc.zmc_integrate(h)
            assert (b.value, b.std, b.flagged_per_level, b.cells_per_level, b.samples) == (
                s.value, s.std, s.flagged_per_level, s.cells_per_level, s.samples), w.name
            assert (b2.value, b2.std) == (b.value, b.std), w.name
            assert b.status == s.status
    finally:
        for h in hs:
            zmc.zmc_destroy(h)


def test_batch_fp64_matches_oracle(zmc):
    ws = mixed_batch()[::3]
    hs = handles(zmc, ws, "fp64")
    try:
        res = zmc.zmc_integrate_batch(hs)
    finally:
        for h in hs:
            zmc.zmc_destroy(h)
    for w, r in zip(ws, res):
        ref = run_oracle(w)
        assert r.flagged_per_level == ref.flagged_per_level, w.name
        assert math.isclose(r.value, ref.value, rel_tol=1e-10, abs_tol=1e-14), (w.name, r.value,
                                                                               ref.value)
        assert math.isclose(r.std, ref.std, rel_tol=1e-10, abs_tol=1e-300), w.name


def test_batch_rejects_mixed_precision(zmc):
    ws = mixed_batch()[:2]
    hs = handles(zmc, ws, "fp64")
    try:
        zmc.zmc_set_precision(hs[1], "fp32_kahan")
        with pytest.raises(zmc.ZmcError) as e:
            zmc.zmc_integrate_batch(hs)
        assert e.value.code == zmc.ZMC_ERR_ARG
    finally:
        for h in hs:
            zmc.zmc_destroy(h)


# ------------------------------------------------------- expressions

def test_expression_reproduces_registry_integrand(zmc):
    w = Workload("sin3", "sin_sum", 3, [0.0] * 3, [10.0] * 3, 4, 301, 5, 2, 2.0, 3)
    a, _ = run_gpu(zmc, w, "fp64", trace=False)
    b, _ = run_gpu(zmc, w.with_(integrand="expr:sin(x[0] + x[1] + x[2])"), "fp64", trace=False)
    assert b.flagged_per_level == a.flagged_per_level
    assert math.isclose(a.value, b.value, rel_tol=1e-12, abs_tol=1e-12)
    # and the expression path against the oracle, level by level
    res, levels = run_gpu(zmc, w.with_(integrand="expr:sin(x[0] + x[1] + x[2])"), "fp64")
    compare_fp64(w, res, levels, run_oracle(w))


EXPR_FP64 = [
    # a step in x0 at p0 times a linear ramp in x1
    Workload("step", "expr:(x[0] < p[0] ? p[1] : 0.0) * (1.0 + x[1])", 2, [0.0, 0.0],
             [1.0, 2.0], 4, 512, 6, 3, 1.0, 11, [0.37, 2.5]),
    # a special function, a conditional, parameters, and C's integer 1/2 (= 0)
    Workload("erf_branch", "expr:erf(x[0] * p[2]) * (x[1] > p[0] ? exp(-x[1]) : p[1])"
             " + fmax(x[2], p[2]) + 1/2", 3, [0.0] * 3, [1.0] * 3, 3, 301, 5, 3, 0.8, 6,
             [0.5, 1.25, 0.3]),
    # logic operators and nested conditionals
    Workload("logic", "expr:(x[0] > 0.25 && x[1] < 0.75) || x[0] + x[1] > 1.5 ? "
             "pow(x[0], 2.0) + 0.5 : (x[1] < 0.1 ? 3.0 : sqrt(x[1]))", 2, [0.0, 0.0],
             [1.0, 1.0], 5, 97, 4, 3, 0.5, 9),
]

EXPR_FP32 = [
    # conditionals continuous at their switch (FP32 rounding of a point near
    # the switch then moves the value by rounding only)
    Workload("erf_knee", "expr:erf(x[0]) * (x[1] > p[0] ? exp(-(x[1] - p[0])) : 1.0)", 2,
             [0.0, 0.0], [1.0, 2.0], 3, 400, 5, 2, 1.0, 4, [0.5]),
    Workload("hinge", "expr:fmax(x[0] - p[0], 0.0) * (x[1] < p[1] ? 1.0 + x[1] : "
             "1.0 + p[1]) + cos(p[2] * x[2])", 3, [0.0] * 3, [1.0] * 3, 3, 256, 6, 2, 1.0, 8,
             [0.4, 0.6, 3.0]),
]


@pytest.mark.parametrize("w", EXPR_FP64, ids=[w.name for w in EXPR_FP64])
def test_expression_with_parameters_and_conditionals_fp64(zmc, w):
    # element by element against the oracle's expression evaluator: sums at
    # 1e-12, identical cell statistics, thresholds and flags, value at 1e-10
    res, levels = run_gpu(zmc, w, "fp64")
    compare_fp64(w, res, levels, run_oracle(w))


@pytest.mark.parametrize("precision", ["fp32_fp64acc", "fp32_kahan"])
@pytest.mark.parametrize("w", EXPR_FP32, ids=[w.name for w in EXPR_FP32])
def test_expression_with_parameters_and_conditionals_fp32(zmc, w, precision):
    res, levels = run_gpu(zmc, w, precision)
    fp32_levels_against_oracle(w, levels, run_oracle(w, fp32_uniforms=True))
    check_decisions_consistent(w, levels, res)


def test_expression_closed_forms(zmc):
    # the step: 2.5 * 0.37 * int_0^2 (1 + x1) dx1; the knee: int_0^1 erf *
    # int_0^2 (x1 > 0.5 ? e^-(x1 - 0.5) : 1)
    step, knee = EXPR_FP64[0], EXPR_FP32[0]
    exact = {"step": 2.5 * 0.37 * 4.0,
             "erf_knee": (math.erf(1.0) + (math.exp(-1.0) - 1.0) / math.sqrt(math.pi))
             * (0.5 + 1.0 - math.exp(-1.5))}
    for w in (step, knee):
        for precision in ("fp64", "fp32_fp64acc"):
            res, _ = run_gpu(zmc, w, precision, trace=False)
            assert abs(res.value - exact[w.name]) <= 3 * res.std, (w.name, precision, res.value,
                                                                   res.std)


def test_expression_matches_closed_form_genz_gauss(zmc):
    a, u = [4.0, 7.0, 2.0], [0.3, 0.6, 0.45]
    expr = "expr:exp(-(p[0]*p[0]*(x[0]-p[3])*(x[0]-p[3]) + p[1]*p[1]*(x[1]-p[4])*(x[1]-p[4])" \
           " + p[2]*p[2]*(x[2]-p[5])*(x[2]-p[5])))"
    w = Workload("gg", expr, 3, [0.0] * 3, [1.0] * 3, 3, 400, 6, 2, 1.0, 4, a + u)
    res, _ = run_gpu(zmc, w, "fp64", trace=False)
    exact = CF.genz_gauss([0.0] * 3, [1.0] * 3, a, u)
    assert abs(res.value - exact) <= 3 * res.std, (res.value, exact, res.std)


def test_expression_compile_error_reports_log(zmc):
    h = zmc.zmc_create(2, [0.0, 0.0], [1.0, 1.0], 2, 16, 2, 1, 1.0, 0)
    try:
        with pytest.raises(zmc.ZmcError) as e:
            zmc.zmc_set_integrand(h, "expr:x[0] + no_such_function(x[1])")
        assert e.value.code == zmc.ZMC_ERR_COMPILE
        assert "no_such_function" in zmc.zmc_last_error(h)
    finally:
        zmc.zmc_destroy(h)


# ------------------------------------------------------- launch shape

@pytest.mark.parametrize("precision", ["fp64", "fp32_kahan"])
def test_results_do_not_depend_on_launch_shape(zmc, precision):
    w = Workload("corner4", "genz_corner", 4, [0.0] * 4, [1.0] * 4, 3, 3001, 6, 3, 0.5, 5,
                 [1.0, 2.0, 3.0, 4.0])
    results = []
    for threads, per_sm in [(0, 0), (64, 1), (128, 2), (256, 0)]:
        it = zmc.Integrator(w.dim, w.lo, w.hi, w.k, w.n, w.trials, w.depth,
                            w.sigma_multiplier, w.seed, w.integrand, w.params,
                            precision=zmc.PRECISIONS[precision])
        try:
            zmc.zmc_set_launch(it.h, threads, per_sm)
            r = it.integrate()
            shape = zmc.zmc_launch_shape(it.h)
            if threads:
                assert shape[0] == threads
        finally:
            it.close()
        results.append((r.value, r.std, r.flagged_per_level, r.cells_per_level))
    assert all(x == results[0] for x in results), results
