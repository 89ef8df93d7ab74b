"""Pins of the oracle's tree search (Sec. 2.1, Fig. 1) against exact cases,
closed forms, a textbook estimator and a brute-force re-derivation."""
import itertools
import math

import numpy as np
import pytest

from oracle import closed_forms as CF


# ------------------------------------------------------------ exact cases

def test_constant_integrand_is_exact(oracle):
    # every trial estimate is c*V exactly, so every spread is 0, nothing is
    # refined and the value is c * vol(domain) with no rounding at all.
    r = oracle.integrate(3, [0.0] * 3, [10.0] * 3, 4, 1000, 5, 3, 2.0, 7,
                         "constant", [2.5], keep_levels=True)
    assert r.value == 2500.0
    assert r.std == 0.0
    assert r.levels_run == 1 and r.flagged_per_level == [0]
    assert r.status == oracle.STATUS_OK
    lv = r.levels[0]
    assert np.all(lv.sums[:, :, 0] == 2500.0)
    assert np.all(lv.spread == 0.0) and lv.theta == 0.0


def test_selection_rule_hand_cases(oracle):
    s = np.array([1.0, 1.0, 3.0, 3.0])
    mu, sigma, theta = oracle.threshold(s, 1.0)
    assert (mu, sigma, theta) == (2.0, 1.0, 3.0)
    # "larger than" the threshold: equality is not flagged
    assert not oracle.select(s, theta, 1, 3).any()
    _, _, theta = oracle.threshold(s, 0.5)
    assert theta == 2.5
    assert oracle.select(s, theta, 1, 3).tolist() == [False, False, True, True]
    # never at the last level
    assert not oracle.select(s, theta, 3, 3).any()
    # all spreads equal: sigma = 0, theta = mu, nothing flagged
    e = np.full(7, 0.3)
    _, sg, th = oracle.threshold(e, 4.0)
    assert sg == 0.0 and not oracle.select(e, th, 1, 2).any()
    # one outlier among eight: mu = 1, sigma = sqrt(7)
    o = np.array([0.0] * 7 + [8.0])
    mu, sigma, theta = oracle.threshold(o, 1.0)
    assert mu == 1.0 and sigma == pytest.approx(math.sqrt(7.0), rel=1e-15)
    assert oracle.select(o, theta, 1, 2).tolist() == [False] * 7 + [True]


def test_margins_hand_cases(oracle):
    # margin_c = |s_c - theta| / theta: the relative distance of a decision
    # from a tie, taken against theta (not mu), the same on both sides
    s = np.array([1.0, 1.0, 3.0, 3.0])
    mu, _, theta = oracle.threshold(s, 0.5)          # mu = 2, theta = 2.5
    assert mu == 2.0 and theta == 2.5
    m = oracle.margins(s, theta)
    assert m.tolist() == [0.6, 0.6, 0.2, 0.2]        # |1 - 2.5| / 2.5, |3 - 2.5| / 2.5
    # an exact tie at theta has margin 0
    assert oracle.margins(np.array([2.5, 0.5]), 2.5).tolist() == [0.0, 0.8]
    # theta <= 0 (every spread 0): no decision is near a tie
    assert np.all(np.isinf(oracle.margins(np.zeros(3), 0.0)))
    # the per-level minimum the oracle reports is that of its own spreads and
    # threshold, and +inf at the last level (no decision is taken there)
    r = oracle.integrate(2, [0.0, 0.0], [1.0, 1.0], 3, 40, 4, 2, 0.5, 3, "genz_gauss",
                         [6.0, 6.0, 0.5, 0.5], keep_levels=True)
    lv = r.levels[0]
    expect = float(np.min(np.abs(lv.spread - lv.theta) / lv.theta))
    assert r.min_margin_per_level[0] == lv.min_margin == expect
    assert r.levels_run == 2 and math.isinf(r.min_margin_per_level[1])


def test_trial_statistics_ddof(oracle):
    sums = np.zeros((2, 3, 2))
    sums[0, :, 0] = [1.0, 2.0, 3.0]
    sums[1, :, 0] = [4.0, 4.0, 4.0]
    est, mean, spread = oracle.cell_statistics(sums, 2.0, 1)
    assert mean.tolist() == [4.0, 8.0]
    assert spread.tolist() == [2.0, 0.0]    # sample std (ddof 1) of 2,4,6


# --------------------------------------------------------------- geometry

def test_level1_order_and_children_tile_the_parent(oracle):
    k, d = 3, 2
    c1 = oracle.level1_cells(k, d)
    assert c1[:4].tolist() == [[0, 0], [1, 0], [2, 0], [0, 1]]   # dim 0 fastest
    parents = c1[[4, 7]]
    kids = oracle.children(parents, k)
    assert kids.shape == (2 * k ** d, d)
    for r, p in enumerate(parents):
        block = kids[r * k ** d:(r + 1) * k ** d]
        # children cover the parent's box exactly once at the finer level
        cells = {tuple(x) for x in block}
        expect = {tuple(k * p + np.array(o)) for o in itertools.product(range(k), repeat=d)}
        assert cells == expect and len(block) == k ** d
        # child `digit` sits at k*c + digits(digit)
        for digit in range(k ** d):
            assert block[digit].tolist() == (k * p + oracle.digits(digit, k, d)).tolist()


def test_depth1_is_the_textbook_stratified_estimator(oracle):
    # Recompute a depth-1 run from the stream words alone: per cell the
    # average of f over all trials and samples, times the cell volume.
    d, k, n, T, seed = 2, 3, 40, 4, 99
    lo, hi = np.array([0.0, -1.0]), np.array([2.0, 3.0])
    r = oracle.integrate(d, lo, hi, k, n, T, 1, 2.0, seed, "sin_sum")
    w = (hi - lo) / k
    total = 0.0
    for q, c in enumerate(oracle.level1_cells(k, d)):
        acc = 0.0
        for t in range(T):
            words = oracle.stream_words(seed, 1, q, t, d, 0, n)
            u = (words.astype(np.float64) + 0.5) / 2.0**32
            x = lo + (c + u) * w
            acc += np.sin(x.sum(axis=1)).sum()
        total += np.prod(w) * acc / (n * T)
    assert r.value == pytest.approx(total, rel=1e-12, abs=1e-14)


# -------------------------------------------------- closed-form agreement

WORKLOADS = [
    ("sin_sum", 3, 0.0, 10.0, [], 4, 1000, 5, 2, 2.0),
    ("sin_sum", 2, -1.0, 4.0, [], 3, 500, 6, 3, 1.0),
    ("gauss_norm", 3, -1.0, 1.0, [0.2], 3, 400, 6, 3, 1.5),
    ("genz_osc", 3, 0.0, 1.0, [0.25, 3.0, 6.0, 9.0], 3, 300, 5, 2, 1.0),
    ("genz_prodpeak", 2, 0.0, 1.0, [4.0, 9.0, 0.3, 0.6], 4, 300, 5, 3, 1.0),
    ("genz_gauss", 3, 0.0, 1.0, [2.0, 6.0, 8.0, 0.5, 0.2, 0.8], 3, 300, 5, 2, 2.0),
    ("genz_corner", 3, 0.0, 1.0, [1.0, 3.0, 4.5], 3, 300, 6, 3, 1.0),
    ("linear", 2, 0.0, 2.0, [1.0, 0.5, -2.0], 4, 200, 5, 2, 1.0),
]


@pytest.mark.parametrize("w", WORKLOADS, ids=[w[0] for w in WORKLOADS])
def test_value_within_five_sigma_of_closed_form(oracle, w):
    name, d, a, b, p, k, n, T, depth, m = w
    lo, hi = [a] * d, [b] * d
    r = oracle.integrate(d, lo, hi, k, n, T, depth, m, 12345, name, p)
    exact = CF.integral(name, lo, hi, p)
    assert r.std > 0
    assert abs(r.value - exact) <= 5 * r.std, (r.value, exact, r.std)
    # and the spread must not be absurdly pessimistic either
    assert r.std < 50 * max(abs(exact), 1e-3)


@pytest.mark.slow
def test_error_coverage(oracle):
    # The error reading (standard errors of the accepted cell means added in
    # quadrature) is fixed statistically: across independent seeds the value
    # falls within 2 std of the closed form about 95% of the time.
    d, k, n, T = 2, 4, 64, 6
    lo, hi = [0.0, 0.0], [3.0, 3.0]
    exact = CF.sin_sum(lo, hi)
    one, two, N = 0, 0, 200
    for seed in range(N):
        r = oracle.integrate(d, lo, hi, k, n, T, 2, 1.0, seed, "sin_sum", threads=1)
        one += abs(r.value - exact) <= r.std
        two += abs(r.value - exact) <= 2 * r.std
    # binomial(200, 0.683) and binomial(200, 0.954) at about 3 sd: an error
    # bar off by sqrt(trials) in either direction fails one of the windows.
    assert 0.58 * N <= one <= 0.79 * N, one
    assert 0.90 * N <= two <= 0.995 * N, two


def test_trial_spread_matches_within_cell_variance(oracle):
    # E[s_c^2] = V^2 Var_cell(f) / n: compare the average of s_c^2 with the
    # within-cell variance estimated from S2 across all cells of one level.
    d, k, n, T = 2, 4, 256, 16
    r = oracle.integrate(d, [0.0, 0.0], [6.0, 6.0], k, n, T, 1, 1.0, 3,
                         "sin_sum", keep_levels=True)
    lv = r.levels[0]
    V = float(np.prod([1.5, 1.5]))
    S1, S2 = lv.sums[:, :, 0], lv.sums[:, :, 1]
    var_f = (S2.sum(1) - S1.sum(1) ** 2 / (n * T)) / (n * T - 1)
    predicted = (V ** 2 * var_f / n).mean()
    observed = (lv.spread ** 2).mean()
    C = lv.spread.size
    # s^2 (T-1)/sigma^2 ~ chi2(T-1): relative sd of the mean ~ sqrt(2/(T-1)/C)
    assert observed == pytest.approx(predicted, rel=5 * math.sqrt(2 / (T - 1) / C))


# ----------------------------------------------------- brute-force tree

def _brute_force_tree(oracle, d, k, n, T, depth, m, seed, name, p, lo, hi):
    """Independent restatement of the tree search over the FULL lattice.

    Every level enumerates all k^(d L) lattice cells; a cell is live when its
    parent was live and flagged.  Live cells are ordered by (slot of the
    parent, child digit).  Decisions use the same rule, applied to the
    spreads of the live cells only.
    """
    lo, hi = np.array(lo), np.array(hi)
    live = {tuple(c): q for q, c in enumerate(
        itertools.product(*[range(k)] * d))}
    # itertools.product varies the LAST index fastest; reorder to dim 0 fastest
    order = sorted(live, key=lambda c: sum(c[i] * k ** i for i in range(d)))
    live = {c: q for q, c in enumerate(order)}
    value_terms, var_terms, flagged_counts = [], [], []
    for L in range(1, depth + 1):
        cells = sorted(live, key=live.get)
        coords = np.array(cells, dtype=np.int64)
        sums = oracle.cell_sums(seed, L, lo, hi, k, n, T, name, p,
                                np.arange(len(cells)), coords)
        V = float(np.prod((hi - lo) / k ** L))
        est = V * sums[:, :, 0] / n
        mean = est.mean(1)
        sd = np.sqrt(((est - mean[:, None]) ** 2).sum(1) / (T - 1))
        mu = sd.sum() / sd.size
        sigma = math.sqrt(((sd - mu) ** 2).sum() / sd.size)
        theta = mu + m * sigma
        flagged = [c for c, s in zip(cells, sd) if L < depth and s > theta]
        flagged_counts.append(len(flagged))
        for c, mval, s in zip(cells, mean, sd):
            if c not in flagged:
                value_terms.append(mval)
                var_terms.append(s * s / T)
        if not flagged:
            break
        nxt = []
        for c in itertools.product(*[range(k ** (L + 1))] * d):
            parent = tuple(x // k for x in c)
            if parent in flagged:
                digit = sum((c[i] % k) * k ** i for i in range(d))
                nxt.append((flagged.index(parent), digit, c))
        live = {c: q for q, (_, _, c) in enumerate(sorted(nxt))}
    return math.fsum(value_terms), math.sqrt(math.fsum(var_terms)), flagged_counts


@pytest.mark.parametrize("d,k,depth,m,seed,name,p", [
    (1, 3, 3, 0.5, 1, "sin_sum", []),
    (2, 2, 3, 0.3, 2, "sin_sum", []),
    (2, 3, 2, 0.0, 3, "genz_gauss", [5.0, 7.0, 0.3, 0.6]),
    (1, 2, 3, 0.0, 4, "genz_corner", [6.0]),
    (2, 2, 3, 1.0, 5, "genz_prodpeak", [8.0, 8.0, 0.5, 0.5]),
])
def test_tree_search_matches_brute_force(oracle, d, k, depth, m, seed, name, p):
    lo, hi = [0.0] * d, [1.0] * d
    n, T = 30, 4
    r = oracle.integrate(d, lo, hi, k, n, T, depth, m, seed, name, p)
    v, s, fl = _brute_force_tree(oracle, d, k, n, T, depth, m, seed, name, p, lo, hi)
    assert r.flagged_per_level == fl
    assert r.value == pytest.approx(v, rel=1e-13, abs=1e-15)
    assert r.std == pytest.approx(s, rel=1e-12, abs=1e-15)
    assert sum(fl) > 0   # the case must actually refine


def test_budget_accepts_level_whole(oracle):
    args = (2, [0.0, 0.0], [1.0, 1.0], 3, 50, 4, 3, 0.0, 11, "genz_gauss",
            [6.0, 6.0, 0.5, 0.5])
    free = oracle.integrate(*args)
    assert free.flagged_per_level[0] > 0
    capped = oracle.integrate(*args, max_cells=free.flagged_per_level[0] * 9 - 1)
    assert capped.status == oracle.STATUS_BUDGET
    assert capped.levels_run == 1 and capped.flagged_per_level == [0]
    # level 1 accepted whole = the depth-1 result
    d1 = oracle.integrate(2, [0.0, 0.0], [1.0, 1.0], 3, 50, 4, 1, 0.0, 11,
                          "genz_gauss", [6.0, 6.0, 0.5, 0.5])
    assert capped.value == d1.value
    capped_s = oracle.integrate(*args, max_samples=9 * 50 * 4)
    assert capped_s.status == oracle.STATUS_BUDGET and capped_s.value == d1.value


def test_fp32_stream_is_an_independent_estimate(oracle):
    # The FP32 stream samples other points (eleven 23-bit fields per pair of blocks):
    # both estimates agree with the closed form and with each other within
    # their errors.
    args = (3, [0.0] * 3, [10.0] * 3, 4, 2000, 5, 1, 2.0, 0, "sin_sum")
    a = oracle.integrate(*args)
    b = oracle.integrate(*args, fp32_uniforms=True)
    exact = CF.sin_sum([0.0] * 3, [10.0] * 3)
    assert a.value != b.value
    assert abs(a.value - exact) <= 5 * a.std and abs(b.value - exact) <= 5 * b.std
    assert abs(a.value - b.value) <= 5 * math.hypot(a.std, b.std)
