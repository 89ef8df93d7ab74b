"""Pins of the oracle's expression evaluator (user integrands with condition
checks and special functions, Sec. 3.3 and Sec. 4): C's precedence,
associativity and integer arithmetic on hand cases; the registry integrands'
formulas (the oracle's C sampler, itself pinned by closed forms) written as
expressions; closed-form integrals of expressions with conditionals,
parameters and special functions."""
import math

import numpy as np
import pytest

from oracle import closed_forms as CF
from oracle.expression import Expression

X = np.array([[0.2, 0.7, 1.5], [0.5, 0.1, -0.25], [0.9, 0.9, 0.0]])


@pytest.mark.parametrize("text,want", [
    ("1 + 2 * 3", 7.0), ("(1 + 2) * 3", 9.0), ("2 - 3 - 4", -5.0), ("8 / 4 / 2", 1.0),
    ("1/2", 0.0), ("-7/2", -3.0), ("7/-2", -3.0), ("1.0/2", 0.5), ("1/2.0", 0.5),
    ("3.0f * 2", 6.0), ("1e2 + .5", 100.5), ("-2 * 3", -6.0), ("- -2", 2.0),
    ("1 ? 2 : 0 ? 3 : 4", 2.0), ("0 ? 2 : 0 ? 3 : 4", 4.0), ("0 ? 2 : 1 ? 3 : 4", 3.0),
    ("!0 + !3", 1.0), ("1 && 0 || 1", 1.0), ("0 || 0 && 1", 0.0), ("1 < 2 == 1", 1.0),
    ("(1 < 2) + (3 <= 3) + (2 > 3) + (2 >= 3) + (4 != 4)", 2.0),
    ("pow(2.0, 10)", 1024.0), ("fmax(1.0, fmin(5.0, 3.0))", 3.0), ("fabs(-2.5)", 2.5),
    ("sqrt(16.0) + exp(0.0) + log(1.0)", 5.0), ("fma(2.0, 3.0, 1.0)", 7.0),
])
def test_constant_expressions_follow_c(text, want):
    assert Expression(text).eval(X).tolist() == [want] * X.shape[0]


def test_coordinates_parameters_and_conditionals():
    p = [0.3, 2.5, -1.0]
    e = Expression("expr:x[0] < p[0] ? p[1] : p[2] * x[1]")
    assert e.eval(X, p).tolist() == [2.5, -0.1, -0.9]
    e = Expression("x[0] > 0.3 && x[1] < 0.5 || x[2] == 0.0")
    assert e.eval(X).tolist() == [0.0, 1.0, 1.0]
    e = Expression("sinf(x[0]) + __expf(x[1]) - erf(x[2])")
    want = [math.sin(a) + math.exp(b) - math.erf(c) for a, b, c in X]
    np.testing.assert_allclose(e.eval(X), want, rtol=1e-15)


@pytest.mark.parametrize("text", ["x[0] +", "(x[0]", "x[0] ? 1", "x[i]", "foo(x[0])",
                                  "x[0] x[1]", "sin(x[0], x[1])", "x[0] % 2"])
def test_malformed_expressions_are_rejected(text):
    with pytest.raises((ValueError, IndexError)):
        Expression(text).eval(X)


def registry_as_expressions(d):
    """Each registry integrand's formula as an expression, with parameters."""
    a = [1.5 + 0.5 * i for i in range(d)]
    u = [0.2 + 0.1 * i for i in range(d)]
    sx = " + ".join("x[%d]" % i for i in range(d))
    dot = " + ".join("p[%d] * x[%d]" % (1 + i, i) for i in range(d))
    prod = " * ".join("1.0 / (1.0 / (p[%d] * p[%d]) + (x[%d] - p[%d]) * (x[%d] - p[%d]))"
                      % (i, i, i, d + i, i, d + i) for i in range(d))
    gsum = " + ".join("p[%d] * p[%d] * (x[%d] - p[%d]) * (x[%d] - p[%d])"
                      % (i, i, i, d + i, i, d + i) for i in range(d))
    corner = " + ".join("p[%d] * x[%d]" % (i, i) for i in range(d))
    r2 = " + ".join("x[%d] * x[%d]" % (i, i) for i in range(d))
    return [
        ("sin_sum", [], "sin(%s)" % sx),
        ("linear", [0.5] + a, "p[0] + %s" % dot),
        ("genz_osc", [0.3] + a, "cos(2.0 * 3.14159265358979323846 * p[0] + %s)" % dot),
        ("genz_prodpeak", a + u, prod),
        ("genz_gauss", a + u, "exp(-(%s))" % gsum),
        ("genz_corner", a, "pow(1.0 + %s, -%d.0)" % (corner, d + 1)),
        ("gauss_norm", [0.3], "pow(sqrt(2.0 * 3.14159265358979323846) * p[0], -%d.0) * "
                              "exp(-(%s) / (2.0 * p[0] * p[0]))" % (d, r2)),
    ]


@pytest.mark.parametrize("d", [1, 3])
def test_registry_formulas_as_expressions(oracle, d):
    # per-(cell, trial) sums of every registry integrand through the C sampler
    # and of the same formula through the evaluator, on the same stream
    lo, hi, k, n, T = [0.0] * d, [1.0] * d, 3, 64, 3
    coords = oracle.level1_cells(k, d)
    slots = np.arange(coords.shape[0])
    for name, params, text in registry_as_expressions(d):
        for fp32 in (False, True):
            ref = oracle.cell_sums(5, 1, lo, hi, k, n, T, name, params, slots, coords,
                                   fp32_uniforms=fp32)
            got = oracle.cell_sums(5, 1, lo, hi, k, n, T, "expr:" + text, params, slots, coords,
                                   fp32_uniforms=fp32)
            np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max(),
                                       err_msg=name)


def test_expression_integrals_match_closed_forms(oracle):
    # a step in x0 at p0 times a ramp in x1: 2.5 * 0.37 * int_0^2 (1 + x1)
    r = oracle.integrate(2, [0.0, 0.0], [1.0, 2.0], 4, 512, 6, 3, 1.0, 11,
                         "expr:(x[0] < p[0] ? p[1] : 0.0) * (1.0 + x[1])", [0.37, 2.5])
    exact = 2.5 * 0.37 * 4.0
    assert abs(r.value - exact) <= 3 * r.std, (r.value, exact, r.std)
    # erf, a conditional continuous at its switch, and a parameter:
    # int_0^1 erf(x0) dx0 * int_0^2 (x1 > 0.5 ? e^-(x1 - 0.5) : 1) dx1
    r = oracle.integrate(2, [0.0, 0.0], [1.0, 2.0], 3, 400, 5, 2, 1.0, 4,
                         "expr:erf(x[0]) * (x[1] > p[0] ? exp(-(x[1] - p[0])) : 1.0)", [0.5])
    exact = (math.erf(1.0) + (math.exp(-1.0) - 1.0) / math.sqrt(math.pi)) * (
        0.5 + 1.0 - math.exp(-1.5))
    assert abs(r.value - exact) <= 3 * r.std, (r.value, exact, r.std)
    # a registry formula as an expression integrates to its closed form
    a, u = [4.0, 7.0], [0.3, 0.6]
    r = oracle.integrate(2, [0.0, 0.0], [1.0, 1.0], 3, 300, 6, 2, 1.0, 4,
                         "expr:exp(-(p[0]*p[0]*(x[0]-p[2])*(x[0]-p[2]) + "
                         "p[1]*p[1]*(x[1]-p[3])*(x[1]-p[3])))", a + u)
    exact = CF.genz_gauss([0.0, 0.0], [1.0, 1.0], a, u)
    assert abs(r.value - exact) <= 3 * r.std, (r.value, exact, r.std)
