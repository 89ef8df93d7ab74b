"""Helpers shared by the GPU parity tests: run one workload through the C ABI
(traced, so every level's data comes back) and through the FP64 oracle, and
compare level by level."""
from __future__ import annotations

import math

import numpy as np

from oracle import zmc_oracle as O

TIE_MARGIN = 1e-9     # decisions closer than this to theta are ties (unpinned)
FP64_SUM_RTOL = 1e-12
FP64_VALUE_RTOL = 1e-10


def run_gpu(zmc, w, precision=None, trace=True, stream=None):
    it = zmc.Integrator(w.dim, w.lo, w.hi, w.k, w.n, w.trials, w.depth, w.sigma_multiplier,
                        w.seed, w.integrand, w.params,
                        precision=zmc.PRECISIONS[precision or w.precision])
    try:
        if w.max_cells is not None or w.max_samples is not None:
            zmc.zmc_set_limits(it.h, w.max_cells or (1 << 24), w.max_samples or (1 << 40))
        it.trace(trace)
        res = it.integrate(stream)
        levels = [it.trace_level(L) for L in range(1, w.depth + 1)] if trace else []
    finally:
        it.close()
    return res, levels


def run_oracle(w, fp32_uniforms=False):
    return O.integrate(w.dim, w.lo, w.hi, w.k, w.n, w.trials, w.depth, w.sigma_multiplier,
                       w.seed, w.integrand, w.params, max_cells=w.max_cells,
                       max_samples=w.max_samples, fp32_uniforms=fp32_uniforms,
                       keep_levels=True)


def sums_tolerance(ref_sums: np.ndarray, n: int, rtol: float) -> np.ndarray:
    """Tolerance per (cell, trial) for (S1, S2).  S1 may cancel to ~0, so its
    scale is sqrt(n * S2) >= sum |f| / sqrt(n) ... >= |S1|; S2 is relative."""
    scale1 = np.sqrt(n * np.abs(ref_sums[..., 1])) + np.abs(ref_sums[..., 0])
    tol = np.empty_like(ref_sums)
    tol[..., 0] = rtol * scale1 + 1e-300
    tol[..., 1] = rtol * np.abs(ref_sums[..., 1]) + 1e-300
    return tol


def spread_tolerance(ref_sums: np.ndarray, volume: float, n: int, rtol: float) -> np.ndarray:
    """Tolerance per cell of its sample spread s (ddof 1 over the T trial
    estimates I_t = V S1_t / n, Sec. 2.1) induced by the allowed error of the
    trials' sums: s moves by at most sqrt(T / (T - 1)) times the largest
    change of an I_t, and each I_t carries a few ulps of its own rounding.
    Relative to s itself this is large where the trials agree closely (s
    then is a difference of nearly equal numbers)."""
    T = ref_sums.shape[1]
    tol1 = sums_tolerance(ref_sums, n, rtol)[..., 0]
    est = volume * np.abs(ref_sums[..., 0]) / n
    return math.sqrt(T / (T - 1)) * (volume / n * tol1.max(axis=1)
                                      + 4 * np.finfo(np.float64).eps * est.max(axis=1))


def compare_fp64(w, res, levels, ref, check_sums=True):
    """Exact decisions and FP64 tolerances, level by level."""
    assert res.levels_run == ref.levels_run, (res.levels_run, ref.levels_run)
    assert res.status == ref.status, (res.status, ref.status)
    for L, (g, r) in enumerate(zip(levels, ref.levels), start=1):
        assert g["cells"] == r.coords.shape[0], L
        if check_sums:
            err = np.abs(g["sums"] - r.sums)
            assert np.all(err <= sums_tolerance(r.sums, w.n, FP64_SUM_RTOL)), (
                L, float(err.max()))
        np.testing.assert_allclose(g["cell_stats"][:, 0], r.mean, rtol=1e-11,
                                   atol=1e-11 * np.abs(r.mean).max() + 1e-300)
        volume = math.prod((b - a) / w.k ** L for a, b in zip(w.lo, w.hi))
        spread_err = np.abs(g["cell_stats"][:, 1] - r.spread)
        bound = np.maximum(1e-10 * r.spread, spread_tolerance(r.sums, volume, w.n,
                                                              FP64_SUM_RTOL)) + 1e-300
        assert np.all(spread_err <= bound), (L, float((spread_err / bound).max()))
        # a cell whose trial sums are identical has spread 0 exactly
        same = np.all(g["sums"][:, :, 0] == g["sums"][:, :1, 0], axis=1)
        assert np.all(g["cell_stats"][same, 1] == 0.0), L
        assert math.isclose(g["theta"], r.theta, rel_tol=1e-10, abs_tol=1e-300), L
        if r.min_margin < TIE_MARGIN:
            raise AssertionError("tie (unpinned): level %d margin %g" % (L, r.min_margin))
        flagged = r.coords[r.flags]
        assert g["flagged"] == flagged.shape[0], (L, g["flagged"], flagged.shape[0])
        assert np.array_equal(g["parents_out"].astype(np.int64), flagged), L
    assert res.flagged_per_level == ref.flagged_per_level
    assert res.cells_per_level == ref.cells_per_level
    assert res.samples == ref.samples and res.cells_evaluated == ref.cells_evaluated
    assert math.isclose(res.value, ref.value, rel_tol=FP64_VALUE_RTOL,
                        abs_tol=FP64_VALUE_RTOL * 1e-300), (res.value, ref.value)
    assert math.isclose(res.std, ref.std, rel_tol=FP64_VALUE_RTOL, abs_tol=1e-300), (
        res.std, ref.std)


def level_coords(w, levels):
    """Lattice coordinates of every traced level's cells, rebuilt on the host
    from the GPU's own parent lists (children of the r-th parent in order)."""
    coords = [O.level1_cells(w.k, w.dim)]
    for g in levels[:-1]:
        if g["flagged"] == 0:
            break
        coords.append(O.children(g["parents_out"].astype(np.int64), w.k))
    return coords


def check_decisions_consistent(w, levels, res):
    """For results whose sums are not bit-comparable (FP32 modes, full sizes):
    the GPU's threshold and flags must follow from the GPU's own spreads."""
    coords = level_coords(w, levels)
    for L, g in enumerate(levels, start=1):
        if g["cells"] == 0:
            break
        s = g["cell_stats"][:, 1]
        mu, sigma = s.mean(), s.std()
        assert math.isclose(g["mu"], mu, rel_tol=1e-9)
        assert math.isclose(g["sigma"], sigma, rel_tol=1e-9, abs_tol=1e-12 * mu)
        theta = mu + w.sigma_multiplier * sigma
        assert math.isclose(g["theta"], theta, rel_tol=1e-9)
        if L < w.depth and g["flagged"] > 0:
            flags = s > g["theta"]
            expect = coords[L - 1][flags]
            assert np.array_equal(g["parents_out"].astype(np.int64), expect), L
    # kernel (c): the value is the sum of the accepted cells' means
    acc_mean, acc_var = [], []
    for L, g in enumerate(levels, start=1):
        if g["cells"] == 0:
            break
        s = g["cell_stats"]
        keep = np.ones(g["cells"], dtype=bool)
        if g["flagged"] > 0:
            keep = ~(s[:, 1] > g["theta"])
        acc_mean.extend(s[keep, 0].tolist())
        acc_var.extend((s[keep, 1] ** 2 / w.trials).tolist())
    assert math.isclose(res.value, math.fsum(acc_mean), rel_tol=1e-12,
                        abs_tol=1e-13 * max(1.0, sum(abs(x) for x in acc_mean)))
    assert math.isclose(res.std, math.sqrt(math.fsum(acc_var)), rel_tol=1e-12)


FP32_SUM_RTOL = 2e-5
# FP32 evaluation moves a spread by about FP32_SUM_RTOL relative: a decision
# whose oracle margin is below this may legitimately go the other way.
FP32_DECISION_MARGIN = 1e-3


def fp32_levels_against_oracle(w, levels, ref):
    """Every level's sums against the oracle on the same (FP32-stream) points
    of the kernel's own cells; the kernel's flags against the oracle's while
    the two trees agree.  Returns the number of divergent decisions (each
    within FP32_DECISION_MARGIN of the oracle's threshold)."""
    coords = level_coords(w, levels)
    divergent = 0
    for L, g in enumerate(levels, start=1):
        if g["cells"] == 0:
            break
        sums = O.cell_sums(w.seed, L, w.lo, w.hi, w.k, w.n, w.trials, w.integrand, w.params,
                           np.arange(g["cells"]), coords[L - 1], fp32_uniforms=True)
        err = np.abs(g["sums"] - sums)
        assert np.all(err <= sums_tolerance(sums, w.n, FP32_SUM_RTOL)), (L, float(err.max()))
        if divergent == 0 and L <= len(ref.levels) and np.array_equal(ref.levels[L - 1].coords,
                                                                      coords[L - 1]):
            r = ref.levels[L - 1]
            flagged = {tuple(c) for c in g["parents_out"].astype(np.int64)}
            mine = np.array([tuple(c) in flagged for c in coords[L - 1]], dtype=bool)
            differ = mine != r.flags
            m = O.margins(r.spread, r.theta)
            assert np.all(m[differ] < FP32_DECISION_MARGIN), (L, float(m[differ].max()))
            divergent += int(differ.sum())
    return divergent
