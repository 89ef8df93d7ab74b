"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 mode: Philox words bit-exact; per-(cell, trial) sums within 1e-12
relative; identical selection decisions (same flagged cells, same order);
final value and error within 1e-10 relative.  FP32 modes: per-(cell, trial)
sums of every level within the FP32 evaluation tolerance of the oracle run on
the same (23-bit) uniforms, decisions consistent with the kernel's own
statistics and equal to the oracle's except within FP32's reach of a tie, and
the value within 3 standard deviations of the closed form.
"""
import math

import numpy as np
import pytest

from oracle import closed_forms as CF
from oracle import zmc_oracle as O
from paper_1902_07916_gb300.workloads import Workload, sin3d

from parity import (check_decisions_consistent, compare_fp64, fp32_levels_against_oracle,
                    run_gpu, run_oracle, sums_tolerance)

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


# ------------------------------------------------------------- generator

@pytest.mark.parametrize("seed,ctr", [
    (0, (0, 0, 0, 0)), (0x123456789ABCDEF0, (7, 3, 11, 2)),
    (2**64 - 1, (0xFFFFFFF0, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF)),
    (42, (1 << 31, 5, 4095, 1)),
])
def test_philox_words_bit_exact(zmc, seed, ctr):
    import torch
    count = 1000   # crosses the 2^32 wrap of counter word 0 for the third case
    out = torch.zeros(4 * count, dtype=torch.int32, device="cuda")
    zmc.zmc_philox_words(seed, *ctr, count, out.data_ptr(),
                         torch.cuda.current_stream())
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32).reshape(count, 4)
    key = O.seed_key(seed)
    for b in list(range(0, count, 37)) + [count - 1]:
        c = ((ctr[0] + b) & 0xFFFFFFFF, ctr[1], ctr[2], ctr[3])
        assert np.array_equal(got[b], O.philox4x32_10(c, key)), b


@pytest.mark.parametrize("mode", ["fp64", "fp32_fp64acc"])
@pytest.mark.parametrize("seed,level,slot,trial,dim,first,count", [
    (0, 1, 0, 0, 1, 0, 97), (0xC0FFEE, 2, 12345, 7, 6, 3, 211),
    (2**64 - 1, 4, 2**32 - 1, 2**32 - 1, 16, 1001, 64), (7, 3, 5, 1, 9, 0, 5),
])
def test_uniforms_bit_exact(zmc, mode, seed, level, slot, trial, dim, first, count):
    # both streams (four 32-bit words per block / eleven 23-bit fields per
    # pair of blocks), for
    # ragged starting points and every dimension, against the oracle
    import torch
    out = torch.full((count * dim,), float("nan"), dtype=torch.float64, device="cuda")
    zmc.zmc_uniforms(seed, level, slot, trial, dim, mode, first, count, out.data_ptr(),
                     torch.cuda.current_stream())
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(count, dim)
    ref = O.stream_uniforms(seed, level, slot, trial, dim, mode != "fp64", first, count)
    assert np.array_equal(got, ref)


# ---------------------------------------------------- FP64 full parity

def W(name, integrand, d, a, b, k, n, T, depth, m, seed, params=(), **kw):
    return Workload(name, integrand, d, [a] * d, [b] * d, k, n, T, depth, m, seed,
                    list(params), **kw)


FP64_CASES = [
    sin3d(),
    W("sin1d_ragged", "sin_sum", 1, -2.0, 3.0, 5, 7, 3, 3, 0.5, 11),
    W("gauss2_n2", "genz_gauss", 2, 0.0, 1.0, 3, 2, 2, 4, 0.0, 5, [6.0, 3.0, 0.4, 0.7]),
    W("corner5", "genz_corner", 5, 0.0, 1.0, 2, 33, 4, 3, 0.5, 3, [1.0, 2.0, 3.0, 4.0, 5.0]),
    W("linear16", "linear", 16, -1.0, 1.0, 2, 9, 2, 1, 1.0, 9,
      [0.5] + [0.1 * i for i in range(16)]),
    W("prodpeak4", "genz_prodpeak", 4, 0.0, 1.0, 3, 101, 6, 3, 1.0, 4,
      [5.0, 7.0, 2.0, 9.0, 0.3, 0.5, 0.7, 0.1]),
    W("gaussnorm3", "gauss_norm", 3, -1.0, 1.0, 4, 64, 4, 3, 1.0, 8, [0.2]),
    W("osc3", "genz_osc", 3, 0.0, 1.0, 3, 50, 5, 3, 0.8, 6, [0.3, 4.0, 8.0, 2.0]),
    W("sin6_tiles", "sin_sum", 6, 0.0, 10.0, 4, 256, 10, 2, 1.5, 2),
    # Level sizes around the selection kernels' CTA counts (one CTA per 1024
    # cells for flag and compaction, per 4096 (cell, trial) sums for the
    # statistics, at most the 256-CTA grid): exactly one CTA, two CTAs with
    # an uneven split, twelve, and the capped grid with a short last chunk.
    W("sel_1024", "genz_osc", 2, 0.0, 1.0, 32, 40, 4, 2, 1.0, 21, [0.3, 4.0, 8.0]),
    W("sel_1089", "genz_osc", 2, 0.0, 1.0, 33, 40, 4, 2, 1.0, 22, [0.3, 4.0, 8.0]),
    W("sel_12167", "genz_gauss", 3, 0.0, 1.0, 23, 24, 4, 1, 1.5, 23,
      [6.0, 3.0, 5.0, 0.4, 0.7, 0.5]),
    W("sel_270400", "genz_corner", 2, 0.0, 1.0, 520, 8, 2, 1, 1.0, 24, [3.0, 5.0]),
    # The FP64 sine of a sum takes an integer sum of the Philox words when
    # every dimension has the same width (a cube): a box of unequal widths
    # keeps the per-dimension FMAs, a 9-D cube runs the integer path past the
    # 8-way unrolled dimension loop.
    Workload("sin3_box", "sin_sum", 3, [0.0, -1.0, 2.0], [10.0, 4.0, 3.0], 4, 257, 4, 2, 1.0,
             31),
    W("sin9_cube", "sin_sum", 9, 0.0, 2.0, 2, 64, 4, 2, 1.5, 32),
]


@pytest.mark.parametrize("w", FP64_CASES, ids=[w.name for w in FP64_CASES])
def test_fp64_matches_oracle(zmc, w):
    res, levels = run_gpu(zmc, w, "fp64")
    ref = run_oracle(w)
    compare_fp64(w, res, levels, ref)


def test_fp64_graph_replay_matches_trace(zmc):
    # The production path (captured graph, no per-level sync) gives bit-for-bit
    # the result of the traced path, run after run.
    w = FP64_CASES[3]
    traced, _ = run_gpu(zmc, w, "fp64", trace=True)
    it = zmc.Integrator(w.dim, w.lo, w.hi, w.k, w.n, w.trials, w.depth, w.sigma_multiplier,
                        w.seed, w.integrand, w.params)
    try:
        for _ in range(3):
            r = it.integrate()
            assert (r.value, r.std, r.flagged_per_level) == (
                traced.value, traced.std, traced.flagged_per_level)
    finally:
        it.close()


def test_constant_integrand_exact(zmc):
    w = W("const", "constant", 3, 0.0, 10.0, 4, 1000, 5, 3, 2.0, 7, [2.5])
    for prec in ("fp64", "fp32_fp64acc", "fp32_kahan"):
        res, _ = run_gpu(zmc, w, prec, trace=False)
        assert res.value == 2500.0 and res.std == 0.0, prec
        assert res.levels_run == 1 and res.flagged_per_level == [0]


def test_budget_rule_matches_oracle(zmc):
    base = W("budget", "genz_gauss", 2, 0.0, 1.0, 3, 50, 4, 3, 0.0, 11, [6.0, 6.0, 0.5, 0.5])
    free = run_oracle(base)
    assert free.flagged_per_level[0] > 0
    for kw in ({"max_cells": free.flagged_per_level[0] * 9 - 1},
               {"max_samples": 9 * 50 * 4 + 1}):
        w = base.with_(**kw)
        res, levels = run_gpu(zmc, w, "fp64")
        ref = run_oracle(w)
        assert ref.status == O.STATUS_BUDGET
        assert res.status == zmc.ZMC_ERR_BUDGET
        compare_fp64(w, res, levels, ref)


def test_nonfinite_integrand_is_reported(zmc):
    # (sqrt(2 pi) s)^-d overflows for s = 1e-200 and exp(...) underflows: inf * 0
    w = W("nan", "gauss_norm", 3, -1.0, 1.0, 2, 16, 2, 2, 1.0, 1, [1e-200])
    res, _ = run_gpu(zmc, w, "fp64", trace=False)
    assert res.status == zmc.ZMC_ERR_NONFINITE


# ---------------------------------------------------------- FP32 modes

FP32_CASES = [
    (sin3d(), None),
    (W("gaussnorm3", "gauss_norm", 3, -1.0, 1.0, 4, 256, 6, 3, 1.0, 8, [0.2]), None),
    (W("corner5", "genz_corner", 5, 0.0, 1.0, 2, 129, 8, 2, 0.5, 3, [1.0, 2.0, 3.0, 4.0, 5.0]),
     None),
    (W("prodpeak3", "genz_prodpeak", 3, 0.0, 1.0, 3, 257, 6, 2, 1.0, 4,
       [5.0, 7.0, 2.0, 0.3, 0.5, 0.7]), None),
    # the high dimensions have their own (fully unrolled) sample loops
    (W("osc10", "genz_osc", 10, 0.0, 1.0, 2, 96, 4, 2, 1.0, 5,
       [0.3] + [0.5 + 0.1 * i for i in range(10)]), None),
    (W("sin12", "sin_sum", 12, 0.0, 1.0, 2, 64, 4, 1, 1.0, 6), None),
    (W("genzgauss16", "genz_gauss", 16, 0.0, 1.0, 2, 16, 3, 1, 1.0, 7,
       [0.8] * 16 + [0.4 + 0.01 * i for i in range(16)]), None),
    (W("linear9", "linear", 9, -1.0, 2.0, 3, 41, 4, 1, 1.0, 8,
       [0.5] + [0.2 * i - 0.7 for i in range(9)]), None),
    # tiles of 64..1023 groups on small levels (one tile per warp)
    (W("sin6_seg8", "sin_sum", 6, 0.0, 1.0, 4, 640, 8, 1, 1.0, 13), None),
    (W("genzgauss5_seg16", "genz_gauss", 5, 0.0, 1.0, 5, 600, 8, 1, 1.0, 14,
       [3.0, 4.0, 5.0, 6.0, 7.0, 0.3, 0.4, 0.5, 0.6, 0.7]), None),
]


@pytest.mark.parametrize("prec", ["fp32_fp64acc", "fp32_kahan"])
@pytest.mark.parametrize("w,_", FP32_CASES, ids=[c[0].name for c in FP32_CASES])
def test_fp32_modes_within_stated_tolerance(zmc, w, _, prec):
    res, levels = run_gpu(zmc, w, prec)
    ref = run_oracle(w, fp32_uniforms=True)
    # every level's sums: FP32 points and integrand against FP64 on the same
    # uniforms; decisions consistent with the kernel's own spreads and, where
    # the trees agree, the oracle's except within FP32's reach of a tie
    fp32_levels_against_oracle(w, levels, ref)
    check_decisions_consistent(w, levels, res)
    exact = CF.integral(w.integrand, w.lo, w.hi, w.params)
    assert abs(res.value - exact) <= 3 * res.std, (res.value, exact, res.std)


@pytest.mark.parametrize("prec", ["fp32_fp64acc", "fp32_kahan"])
def test_fp32_modes_keep_values_below_fp32_range(zmc, prec):
    """Eq. (2) with a narrow peak (sigma 0.005 in 5-D): every level-1 value
    lies far below FP32's range (the largest tile sum is ~1e-78), so only the
    log2-domain evaluation of the FP32 modes sees the cell that holds the
    peak and refines it.  Against the FP64 oracle on the same (FP32-stream)
    points: the same cells and flags at every level, sums within the FP32
    exponent's precision, and the same value and error."""
    s = 0.005
    w = Workload("gauss5_narrow", "gauss_norm", 5, [-1.0] * 5, [1.0] * 5, 3, 400, 4, 3, 2.0, 7,
                 [s])
    res, levels = run_gpu(zmc, w, prec)
    ref = run_oracle(w, fp32_uniforms=True)
    C = (math.sqrt(2 * math.pi) * s) ** -5
    assert 0.0 < ref.levels[0].sums[..., 0].max() < 1e-38      # the range FP32 does not have
    assert ref.flagged_per_level[0] == 1
    assert res.levels_run == ref.levels_run
    assert res.flagged_per_level == ref.flagged_per_level
    for L, (g, r) in enumerate(zip(levels, ref.levels), start=1):
        assert g["cells"] == r.coords.shape[0], L
        # FP32 evaluation of exp(E), E = -|x|^2 / (2 s^2): the exponent's own
        # rounding, |E| 2^-22, and the coordinates' (each off by up to
        # 2^-22 max|x| through the FP32 cell coefficients) times the
        # exponent's gradient |x| / s^2 = sqrt(2 |E|) / s, in d dimensions.
        # A tile's largest value has |E| <= |ln(S1 / (n C))|.
        s1 = r.sums[..., 0]
        pos = s1 > 0
        lnE = np.zeros_like(s1)
        lnE[pos] = np.abs(np.log(s1[pos]) - math.log(w.n * C))
        rtol = 2e-5 + 2.0 ** -22 * (lnE + w.dim * 1.0 * np.sqrt(2 * lnE) / s)
        err = np.abs(g["sums"][..., 0] - s1)
        assert np.all(err <= rtol * s1 + 1e-300), (L, float(np.max(err / (s1 + 1e-300))))
        assert np.all((g["sums"][..., 0] > 0) == pos), L
    assert math.isclose(res.value, ref.value, rel_tol=1e-3), (res.value, ref.value)
    assert math.isclose(res.std, ref.std, rel_tol=1e-2), (res.std, ref.std)


@pytest.mark.parametrize("prec", ["fp32_fp64acc", "fp32_kahan"])
def test_fp32_sine_of_large_arguments(zmc, prec):
    """sin(x1 + x2 + x3) on [3000, 3010]^3: arguments near 9000 rad (1430
    turns).  The FP32 modes fold the argument in turns and reduce it by
    t - rint(t), exact for any float; what remains is FP32's rounding of the
    argument itself, (d + 2) ulp of |t| at most, times 2 pi.  Level-1 sums
    against the oracle on the same points within n times that, identical
    flags, value within the same bound."""
    w = Workload("sin3_far", "sin_sum", 3, [3000.0] * 3, [3010.0] * 3, 4, 500, 4, 2, 2.0, 3)
    res, levels = run_gpu(zmc, w, prec)
    ref = run_oracle(w, fp32_uniforms=True)
    t_max = sum(w.hi) / (2 * math.pi)
    e_point = (w.dim + 2) * 2.0 ** -24 * t_max * 2 * math.pi
    err = np.abs(levels[0]["sums"][..., 0] - ref.levels[0].sums[..., 0])
    assert np.all(err <= w.n * e_point), (float(err.max()), w.n * e_point)
    assert res.flagged_per_level == ref.flagged_per_level
    exact = CF.integral(w.integrand, w.lo, w.hi, w.params)
    assert abs(res.value - exact) <= 3 * res.std, (res.value, exact, res.std)


@pytest.mark.parametrize("prec", ["fp64", "fp32_fp64acc"])
def test_lane_tiles_on_a_large_level(zmc, prec):
    """A level of 373,248 tiles of 320 (FP64) or 256 (FP32) point groups: the
    sampling kernel runs 32 whole tiles per warp, one per lane, with no warp
    reduction.  FP64: every sum, statistic and flag against the oracle; FP32:
    sums against the oracle on the same points, consistent decisions."""
    w = W("sin6_lanes", "sin_sum", 6, 0.0, 1.0, 6, 1280, 8, 1, 1.0, 12)
    if prec == "fp64":
        res, levels = run_gpu(zmc, w, prec)
        compare_fp64(w, res, levels, run_oracle(w))
    else:
        res, levels = run_gpu(zmc, w, prec)
        ref = run_oracle(w, fp32_uniforms=True)
        err = np.abs(levels[0]["sums"] - ref.levels[0].sums)
        assert np.all(err <= sums_tolerance(ref.levels[0].sums, w.n, 2e-5)), float(err.max())
        check_decisions_consistent(w, levels, res)
