"""FP64 CPU oracle for stratified sampling with heuristic tree search.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the product library
never calls it.  It shares no code with the CUDA path.

The method (ZMCintegral, arXiv 1902.07916, Sec. 2.1 and Fig. 1):

1. The domain is split into equal hypercube cells (k per dimension, so k^d
   cells at level 1).
2. In every cell the integral is estimated by direct Monte Carlo, and that
   estimate is repeated independently ``trials`` (the paper's n1) times.
3. For every cell the mean and standard deviation of those estimates are
   taken.
4. A threshold is formed from the mean and standard deviation of all the
   cells' standard deviations; a cell whose standard deviation is larger
   than it is split again into k^d equal children (next level), the others
   are accepted.  A new threshold is set at every level.
5. This stops when no cell is flagged or the maximal depth is reached (depth
   1: the domain is divided once and never refined).
6. The accepted cells' means are summed into the integral; their standard
   deviations are collected into its error.

Readings of points the paper leaves open (each is also listed with the design
notes of the repository):

* k is per dimension (the experiments of Sec. 3 state their counts per dimension).
* Cells are numbered row-major with dimension 0 fastest; children of the
  r-th flagged parent (in work-list order) take slots r*k^d + digit, where
  digit = sum_i digit_i k^i and the child's lattice coordinate is
  k*c_i + digit_i.
* Per-cell spread: sample standard deviation over trials (ddof 1).
* Threshold: theta_L = mu_L + m * sigma_L with mu_L, sigma_L the mean and
  population standard deviation (ddof 0) of the level's cell spreads
  (the five-sigma criterion of Sec. 3.1 read as mu + 5 sigma).  A cell is flagged
  when its spread is strictly larger than theta_L, and never at the last level.
* Error: std = sqrt(sum over accepted cells of s_c^2 / trials), i.e. the
  standard errors of the accepted cell means added in quadrature.
  Parity unpinned by the paper (it gives no formula); pinned statistically
  by the coverage tests.
* Budget: if refining level L would make level L+1 larger than
  ``max_cells`` cells, or the run larger than ``max_samples`` samples, level
  L is accepted whole and the run ends with status BUDGET.

The Monte Carlo sums are computed by the C sampler next to this file
(``sampler.c``); everything above them is written out here in numpy, in the
order of the steps above.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

import numpy as np

STATUS_OK = 0
STATUS_BUDGET = 3

# Integrand names and the sampler's numbering of them.
INTEGRANDS = {
    "constant": 0,
    "linear": 1,
    "sin_sum": 2,
    "gauss_norm": 3,
    "genz_osc": 4,
    "genz_prodpeak": 5,
    "genz_gauss": 6,
    "genz_corner": 7,
}

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


def _load():
    global _lib
    if _lib is None:
        from . import build as _build
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.zmc_oracle_philox4x32_10.argtypes = [
            ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
            ctypes.POINTER(ctypes.c_uint32)]
        lib.zmc_oracle_philox4x32_10.restype = None
        lib.zmc_oracle_uniform64.argtypes = [ctypes.c_uint32]
        lib.zmc_oracle_uniform64.restype = ctypes.c_double
        lib.zmc_oracle_field23.argtypes = [ctypes.POINTER(ctypes.c_uint32), ctypes.c_int]
        lib.zmc_oracle_field23.restype = ctypes.c_uint32
        lib.zmc_oracle_field_uniform.argtypes = [ctypes.c_uint32]
        lib.zmc_oracle_field_uniform.restype = ctypes.c_double
        lib.zmc_oracle_pair_field.argtypes = [ctypes.POINTER(ctypes.c_uint32),
                                              ctypes.POINTER(ctypes.c_uint32), ctypes.c_int]
        lib.zmc_oracle_pair_field.restype = ctypes.c_uint32
        lib.zmc_oracle_stream_uniforms.argtypes = [
            ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int,
            ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]
        lib.zmc_oracle_stream_uniforms.restype = None
        lib.zmc_oracle_integrand.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
            ctypes.POINTER(ctypes.c_double)]
        lib.zmc_oracle_integrand.restype = ctypes.c_double
        lib.zmc_oracle_stream_words.argtypes = [
            ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32,
            ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
            ctypes.POINTER(ctypes.c_uint32)]
        lib.zmc_oracle_stream_words.restype = None
        lib.zmc_oracle_cell_sums.argtypes = [
            ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
            ctypes.c_int64, ctypes.c_int, ctypes.c_int,
            ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
            ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_int64),
            ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        lib.zmc_oracle_cell_sums.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


# ------------------------------------------------------------- primitives

def philox4x32_10(counter, key) -> np.ndarray:
    """One Philox4x32-10 block (SC'11 definition) -> 4 uint32 words."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in counter])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    out = (ctypes.c_uint32 * 4)()
    lib.zmc_oracle_philox4x32_10(c, k, out)
    return np.array(list(out), dtype=np.uint32)


def seed_key(seed: int):
    """Philox key of a 64-bit seed: (low word, high word)."""
    return (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


def stream_words(seed: int, level: int, slot: int, trial: int, d: int,
                 s0: int, count: int) -> np.ndarray:
    """Words of the (level, slot, trial) stream, shape (count, d)."""
    lib = _load()
    out = np.zeros(count * d, dtype=np.uint32)
    lib.zmc_oracle_stream_words(seed, level, slot, trial, d, s0, count,
                                _ptr(out, ctypes.c_uint32))
    return out.reshape(count, d)


def uniform64(w: int) -> float:
    """(w + 1/2) / 2^32: the FP64 uniform of one word."""
    return _load().zmc_oracle_uniform64(int(w))


def field23(block, f: int) -> int:
    """Bits [23 f, 23 f + 23) of a Philox block read as a 128-bit integer."""
    w = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in block])
    return _load().zmc_oracle_field23(w, int(f))


def pair_field(block_a, block_b, f: int) -> int:
    """Field f (0..10) of a pair of blocks in the FP32 stream: fields 0..4 of
    the first block, 5..9 of the second, and bits 115..127 of the first with
    bits 115..124 of the second above them."""
    a = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in block_a])
    b = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in block_b])
    return _load().zmc_oracle_pair_field(a, b, int(f))


def field_uniform(field: int) -> float:
    """(f + 1/2) / 2^23: the FP32-stream uniform of a 23-bit field."""
    return _load().zmc_oracle_field_uniform(int(field))


def stream_uniforms(seed: int, level: int, slot: int, trial: int, d: int, fp32: bool,
                    s0: int, count: int) -> np.ndarray:
    """Uniforms of points [s0, s0 + count) of the (level, slot, trial) stream,
    shape (count, d): the FP64 stream (four 32-bit words per block) or the
    FP32 stream (eleven 23-bit fields per pair of blocks)."""
    lib = _load()
    out = np.zeros(count * d, dtype=np.float64)
    lib.zmc_oracle_stream_uniforms(seed, level, slot, trial, d, 1 if fp32 else 0, s0, count,
                                   _ptr(out, ctypes.c_double))
    return out.reshape(count, d)


def integrand_value(name: str, x, params) -> float:
    """The integrand at one point, FP64."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    p = np.ascontiguousarray(params if len(params) else [0.0], dtype=np.float64)
    return lib.zmc_oracle_integrand(INTEGRANDS[name], len(x),
                                    _ptr(x, ctypes.c_double),
                                    _ptr(p, ctypes.c_double))


def cell_sums(seed: int, level: int, lo, hi, k: int, n: int, trials: int,
              integrand: str, params, slots, coords, fp32_uniforms=False,
              threads: int | None = None) -> np.ndarray:
    """(S1, S2) per (cell, trial) of one level: array (cells, trials, 2).

    ``slots`` are the cells' work-list slots q (they select the random
    stream), ``coords`` their lattice coordinates at ``level`` (cells, d).
    """
    if integrand.startswith("expr:"):
        return expression_cell_sums(seed, level, lo, hi, k, n, trials, integrand, params,
                                    slots, coords, fp32_uniforms)
    lib = _load()
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    d = lo.size
    width = np.ascontiguousarray(level_widths(lo, hi, k, level))
    slots = np.ascontiguousarray(slots, dtype=np.uint32)
    coords = np.ascontiguousarray(coords, dtype=np.int64).reshape(-1, d)
    ncell = coords.shape[0]
    p = np.ascontiguousarray(list(params) if len(params) else [0.0],
                             dtype=np.float64)
    out = np.zeros((ncell, trials, 2), dtype=np.float64)
    rc = lib.zmc_oracle_cell_sums(
        seed, level, d, _ptr(lo, ctypes.c_double), _ptr(width, ctypes.c_double),
        n, trials, INTEGRANDS[integrand], _ptr(p, ctypes.c_double), ncell,
        _ptr(slots, ctypes.c_uint32), _ptr(coords, ctypes.c_int64),
        1 if fp32_uniforms else 0, threads or default_threads(),
        _ptr(out, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle sampler rejected its arguments")
    return out


def expression_cell_sums(seed: int, level: int, lo, hi, k: int, n: int, trials: int,
                         expr: str, params, slots, coords, fp32_uniforms=False) -> np.ndarray:
    """(S1, S2) per (cell, trial) for an expression integrand ("expr:..."):
    the same stream, points and sample-order sums as the C sampler, with the
    integrand evaluated by the expression evaluator (expression.py).  For the
    small cases the tests run (numpy over each tile's points)."""
    from .expression import Expression
    e = Expression(expr)
    lo = np.asarray(lo, dtype=np.float64)
    width = level_widths(lo, hi, k, level)
    coords = np.asarray(coords, dtype=np.int64).reshape(-1, lo.size)
    slots = np.asarray(slots, dtype=np.int64)
    out = np.zeros((coords.shape[0], trials, 2), dtype=np.float64)
    for c in range(coords.shape[0]):
        for t in range(trials):
            u = stream_uniforms(seed, level, int(slots[c]), t, lo.size, fp32_uniforms, 0, n)
            x = lo + (coords[c].astype(np.float64) + u) * width     # add, multiply, add
            f = e.eval(x, params)
            out[c, t, 0] = np.cumsum(f)[-1]                          # in sample order
            out[c, t, 1] = np.cumsum(f * f)[-1]
    return out


# ------------------------------------------------------- tree-search steps

def level_widths(lo, hi, k: int, level: int) -> np.ndarray:
    """Cell edge per dimension at a level: (hi - lo) / k^level."""
    return (np.asarray(hi, np.float64) - np.asarray(lo, np.float64)) / float(k ** level)


def digits(index: int | np.ndarray, k: int, d: int) -> np.ndarray:
    """Base-k digits of an index, dimension 0 first (least significant)."""
    index = np.asarray(index, dtype=np.int64)
    out = np.empty(index.shape + (d,), dtype=np.int64)
    rest = index.copy()
    for i in range(d):
        out[..., i] = rest % k
        rest //= k
    return out


def level1_cells(k: int, d: int) -> np.ndarray:
    """All k^d cells of level 1 in row-major order, dimension 0 fastest."""
    return digits(np.arange(k ** d, dtype=np.int64), k, d)


def children(parents: np.ndarray, k: int) -> np.ndarray:
    """Lattice coordinates of the k^d children of each parent, in order.

    Child ``digit`` of parent ``r`` goes to slot r*k^d + digit and has
    coordinate k*c_i + digit_i in dimension i.
    """
    parents = np.asarray(parents, dtype=np.int64)
    d = parents.shape[1]
    dig = digits(np.arange(k ** d, dtype=np.int64), k, d)        # (K, d)
    kids = k * parents[:, None, :] + dig[None, :, :]              # (F, K, d)
    return kids.reshape(-1, d)


def cell_statistics(sums: np.ndarray, volume: float, n: int):
    """Per-cell mean and sample std (ddof 1) of the trial estimates.

    I_{c,t} = V * S1 / n is the direct MC estimate of trial t in cell c.
    """
    est = volume * sums[:, :, 0] / float(n)
    mean = est.mean(axis=1)
    spread = est.std(axis=1, ddof=1)
    return est, mean, spread


def threshold(spread: np.ndarray, m: float):
    """theta = mu + m*sigma over the level's cell spreads (sigma: ddof 0)."""
    mu = float(np.mean(spread))
    sigma = float(np.std(spread))        # two-pass, ddof 0
    return mu, sigma, mu + m * sigma


def select(spread: np.ndarray, theta: float, level: int, depth: int) -> np.ndarray:
    """Flag cells whose spread is strictly larger than theta (never at depth)."""
    if level >= depth:
        return np.zeros(spread.shape, dtype=bool)
    return spread > theta


def margins(spread: np.ndarray, theta: float) -> np.ndarray:
    """|s_c - theta| / theta: how far each decision is from a tie."""
    if theta <= 0.0:
        return np.full(spread.shape, np.inf)
    return np.abs(spread - theta) / theta


@dataclass
class LevelTrace:
    level: int
    coords: np.ndarray      # (C, d) lattice coordinates
    sums: np.ndarray        # (C, T, 2)
    mean: np.ndarray        # (C,)
    spread: np.ndarray      # (C,)
    mu: float
    sigma: float
    theta: float
    flags: np.ndarray       # (C,) bool, after the budget rule
    min_margin: float


@dataclass
class OracleResult:
    value: float
    std: float
    cells_evaluated: int
    samples: int
    levels_run: int
    status: int
    cells_per_level: list = field(default_factory=list)
    flagged_per_level: list = field(default_factory=list)
    theta_per_level: list = field(default_factory=list)
    min_margin_per_level: list = field(default_factory=list)
    levels: list = field(default_factory=list)


def integrate(dim: int, lo, hi, k: int, n: int, trials: int, depth: int,
              sigma_multiplier: float, seed: int, integrand: str, params=(),
              max_cells: int | None = None, max_samples: int | None = None,
              fp32_uniforms: bool = False, keep_levels: bool = False,
              threads: int | None = None) -> OracleResult:
    """Run the whole method, level by level, in FP64."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    assert lo.size == dim and hi.size == dim
    K = k ** dim
    coords = level1_cells(k, dim)
    if max_cells is not None and K > max_cells:
        raise ValueError("level 1 exceeds max_cells")
    if max_samples is not None and K * n * trials > max_samples:
        raise ValueError("level 1 exceeds max_samples")

    accepted_means = []
    accepted_vars = []
    res = OracleResult(0.0, 0.0, 0, 0, 0, STATUS_OK)
    for level in range(1, depth + 1):
        C = coords.shape[0]
        slots = np.arange(C, dtype=np.uint32)
        sums = cell_sums(seed, level, lo, hi, k, n, trials, integrand, params,
                         slots, coords, fp32_uniforms, threads)
        volume = float(np.prod(level_widths(lo, hi, k, level)))
        _, mean, spread = cell_statistics(sums, volume, n)
        mu, sigma, theta = threshold(spread, sigma_multiplier)
        flags = select(spread, theta, level, depth)
        mmin = float(np.min(margins(spread, theta))) if level < depth else math.inf

        res.cells_evaluated += C
        res.samples += C * trials * n
        res.levels_run = level
        F = int(flags.sum())
        if F:
            nxt = F * K
            over_cells = max_cells is not None and nxt > max_cells
            over_samples = (max_samples is not None
                            and res.samples + nxt * n * trials > max_samples)
            if over_cells or over_samples:
                flags = np.zeros_like(flags)
                F = 0
                res.status = STATUS_BUDGET
        res.cells_per_level.append(C)
        res.flagged_per_level.append(F)
        res.theta_per_level.append(theta)
        res.min_margin_per_level.append(mmin)
        if keep_levels:
            res.levels.append(LevelTrace(level, coords.copy(), sums, mean,
                                         spread, mu, sigma, theta, flags.copy(),
                                         mmin))
        keep = ~flags
        accepted_means.extend(mean[keep].tolist())
        accepted_vars.extend((spread[keep] ** 2 / trials).tolist())
        if F == 0:
            break
        coords = children(coords[flags], k)

    res.value = math.fsum(accepted_means)
    res.std = math.sqrt(math.fsum(accepted_vars))
    return res
