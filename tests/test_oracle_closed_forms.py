"""Pins of the closed-form integrals against numerical quadrature, and of the
reading of the paper's two integrands against the results it prints."""
import math
import os

import numpy as np
import pytest

from oracle import closed_forms as CF

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_results.txt")


def _nquad(f, lo, hi):
    integrate = pytest.importorskip("scipy.integrate")
    val, err = integrate.nquad(lambda *x: f(np.array(x)), list(zip(lo, hi)),
                               opts={"epsabs": 1e-12, "epsrel": 1e-11,
                                     "limit": 200})
    return val


CASES = [
    ("sin_sum", [0.0, -1.0], [10.0, 2.5], []),
    ("gauss_norm", [-1.0, -0.3], [1.0, 0.7], [0.3]),
    ("genz_osc", [0.0, 0.0], [1.0, 1.0], [0.3, 4.0, 7.5]),
    ("genz_prodpeak", [0.0, 0.0], [1.0, 1.0], [3.0, 8.0, 0.2, 0.7]),
    ("genz_gauss", [0.0, 0.0], [1.0, 1.0], [2.0, 5.0, 0.4, 0.9]),
    ("genz_corner", [0.0, 0.0], [1.0, 1.0], [0.7, 4.5]),
    ("genz_corner", [0.0, 0.0, 0.0], [1.0, 1.0, 1.0], [1.5, 0.5, 3.0]),
    ("genz_corner", [0.2, 0.1], [0.9, 1.7], [2.0, 1.0]),
    ("constant", [0.0, 1.0], [2.0, 4.0], [2.5]),
    ("linear", [-1.0, 0.0], [1.0, 3.0], [0.5, 2.0, -1.5]),
]


def _pointwise(name, x, p):
    d = x.size
    if name == "sin_sum":
        return math.sin(x.sum())
    if name == "gauss_norm":
        s = p[0]
        return math.exp(-(x ** 2).sum() / (2 * s * s)) / (math.sqrt(2 * math.pi) * s) ** d
    if name == "genz_osc":
        return math.cos(2 * math.pi * p[0] + np.dot(p[1:1 + d], x))
    if name == "genz_prodpeak":
        a, u = np.array(p[:d]), np.array(p[d:])
        return float(np.prod(1.0 / (a ** -2 + (x - u) ** 2)))
    if name == "genz_gauss":
        a, u = np.array(p[:d]), np.array(p[d:])
        return math.exp(-float(((a * (x - u)) ** 2).sum()))
    if name == "genz_corner":
        return (1.0 + np.dot(p[:d], x)) ** (-(d + 1))
    if name == "constant":
        return p[0]
    if name == "linear":
        return p[0] + np.dot(p[1:1 + d], x)
    raise KeyError(name)


@pytest.mark.parametrize("name,lo,hi,p", CASES)
def test_closed_form_matches_quadrature(name, lo, hi, p):
    ref = _nquad(lambda x: _pointwise(name, x, p), lo, hi)
    got = CF.integral(name, lo, hi, p)
    assert got == pytest.approx(ref, rel=1e-8, abs=1e-11)


def test_one_dimensional_textbook_values():
    assert CF.sin_sum([0.0], [10.0]) == pytest.approx(1 - math.cos(10.0), rel=1e-14)
    # erf of a unit-width Gaussian over one standard deviation each side
    assert CF.gauss_norm([-1.0], [1.0], 1.0) == pytest.approx(0.6826894921370859, rel=1e-14)
    # corner peak in 1-D: (1/a) (1 - 1/(1+a))
    a = 3.0
    assert CF.genz_corner([0.0], [1.0], [a]) == pytest.approx((1 - 1 / (1 + a)) / a, rel=1e-15)


def test_workload_closed_forms():
    # sin(x1 + ... + xd) on [0,10]^d for the 3-D and 6-D workloads
    assert CF.sin_sum([0.0] * 3, [10.0] * 3) == pytest.approx(-4.58720932278195, rel=1e-13)
    assert CF.sin_sum([0.0] * 6, [10.0] * 6) == pytest.approx(-49.16507381641946, rel=1e-13)
    # the normalised Gaussian on [-1,1]^9: erf(1/(sigma sqrt 2))^9
    assert CF.gauss_norm([-1.0] * 9, [1.0] * 9, 0.1) == pytest.approx(1.0, abs=1e-15)


def test_corner_peak_against_high_precision():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    a = [0.5 + 0.5 * i for i in range(8)]
    d = len(a)
    total = mpmath.mpf(0)
    for mask in range(1 << d):
        bits = [(mask >> i) & 1 for i in range(d)]
        total += (-1) ** sum(bits) / (1 + mpmath.fsum(mpmath.mpf(a[i]) for i in range(d) if bits[i]))
    ref = total / (mpmath.factorial(d) * mpmath.fprod([mpmath.mpf(x) for x in a]))
    assert CF.genz_corner([0.0] * d, [1.0] * d, a) == pytest.approx(float(ref), rel=1e-14)


def _paper_rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            f, dim, lo, hi, sig, res, std, *src = line.split()
            rows.append((f, int(dim), float(lo), float(hi), float(sig),
                         float(res), float(std), " ".join(src)))
    return rows


@pytest.mark.parametrize("row", _paper_rows(), ids=lambda r: r[7])
def test_paper_results_bracket_closed_form(row):
    f, dim, lo, hi, sig, res, std, src = row
    if f == "f1":
        exact = CF.sin_sum([lo] * dim, [hi] * dim)
    else:
        exact = CF.gauss_norm([lo] * dim, [hi] * dim, sig)
    assert abs(res - exact) <= 3.0 * std, (src, res, exact)
