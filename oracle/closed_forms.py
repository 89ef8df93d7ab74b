"""Closed-form integrals over a box, for pinning the oracle and the kernels.

TEST INFRASTRUCTURE (see zmc_oracle.py).  Pure Python standard library, so it
runs wherever the tests run.  Each integral is over the box prod_i [a_i, b_i]
and is derived analytically from the integrand's definition; none of them
uses the sampler.

* sin(sum x) -- Eq. (1) of the paper, any dimension:
      Im prod_i (e^{i b_i} - e^{i a_i}) / i
* normalised Gaussian -- Eq. (2) of the paper, any dimension and width:
      prod_i [erf(b_i / (sigma sqrt 2)) - erf(a_i / (sigma sqrt 2))] / 2
* Genz oscillatory cos(2 pi u + sum a_i x_i):
      Re e^{2 pi i u} prod_i (e^{i a_i b_i} - e^{i a_i a'_i}) / (i a_i)
* Genz product peak prod_i 1 / (a_i^-2 + (x_i - u_i)^2):
      prod_i a_i [atan(a_i (b_i - u_i)) - atan(a_i (a'_i - u_i))]
* Genz Gaussian exp(-sum a_i^2 (x_i - u_i)^2):
      prod_i sqrt(pi) / (2 a_i) [erf(a_i (b_i - u_i)) - erf(a_i (a'_i - u_i))]
* Genz corner peak (1 + sum a_i x_i)^-(d+1):
      1 / (d! prod a_i) * sum over box vertices v of (-1)^{#upper(v)} / (1 + a.v)
  evaluated in exact rational arithmetic (it cancels badly in floating point).
* constant c: c * vol;  linear b + sum a_i x_i: b vol + sum_i a_i (b_i^2 -
  a_i^2)/2 * prod_{j != i} (b_j - a_j).
"""
from __future__ import annotations

import cmath
import itertools
import math
from fractions import Fraction


def sin_sum(lo, hi) -> float:
    p = complex(1.0, 0.0)
    for a, b in zip(lo, hi):
        p *= (cmath.exp(1j * b) - cmath.exp(1j * a)) / 1j
    return p.imag


def gauss_norm(lo, hi, sigma: float) -> float:
    r = 1.0
    s = sigma * math.sqrt(2.0)
    for a, b in zip(lo, hi):
        r *= 0.5 * (math.erf(b / s) - math.erf(a / s))
    return r


def genz_osc(lo, hi, u1: float, a) -> float:
    p = cmath.exp(2j * math.pi * u1)
    for l, h, ai in zip(lo, hi, a):
        p *= (cmath.exp(1j * ai * h) - cmath.exp(1j * ai * l)) / (1j * ai)
    return p.real


def genz_prodpeak(lo, hi, a, u) -> float:
    r = 1.0
    for l, h, ai, ui in zip(lo, hi, a, u):
        r *= ai * (math.atan(ai * (h - ui)) - math.atan(ai * (l - ui)))
    return r


def genz_gauss(lo, hi, a, u) -> float:
    r = 1.0
    for l, h, ai, ui in zip(lo, hi, a, u):
        r *= math.sqrt(math.pi) / (2.0 * ai) * (math.erf(ai * (h - ui))
                                                - math.erf(ai * (l - ui)))
    return r


def genz_corner(lo, hi, a) -> float:
    """Exact rational evaluation of the vertex sum, rounded once at the end."""
    d = len(a)
    A = [Fraction(x) for x in a]
    L = [Fraction(x) for x in lo]
    H = [Fraction(x) for x in hi]
    total = Fraction(0)
    for upper in itertools.product((0, 1), repeat=d):
        v = [H[i] if upper[i] else L[i] for i in range(d)]
        denom = 1 + sum(A[i] * v[i] for i in range(d))
        if denom <= 0:
            raise ValueError("1 + a.x must stay positive on the box")
        sign = -1 if (sum(upper) % 2) else 1
        total += Fraction(sign) / denom
    prod_a = Fraction(1)
    for x in A:
        prod_a *= x
    return float(total / (math.factorial(d) * prod_a))


def constant(lo, hi, c: float) -> float:
    return c * math.prod(b - a for a, b in zip(lo, hi))


def linear(lo, hi, b0: float, a) -> float:
    edges = [h - l for l, h in zip(lo, hi)]
    vol = math.prod(edges)
    total = b0 * vol
    for i, (l, h, ai) in enumerate(zip(lo, hi, a)):
        rest = math.prod(edges[j] for j in range(len(edges)) if j != i)
        total += ai * (h * h - l * l) / 2.0 * rest
    return total


def integral(name: str, lo, hi, params) -> float:
    """Closed form of a registry integrand (same parameter layout)."""
    d = len(lo)
    p = list(params)
    if name == "constant":
        return constant(lo, hi, p[0])
    if name == "linear":
        return linear(lo, hi, p[0], p[1:1 + d])
    if name == "sin_sum":
        return sin_sum(lo, hi)
    if name == "gauss_norm":
        return gauss_norm(lo, hi, p[0])
    if name == "genz_osc":
        return genz_osc(lo, hi, p[0], p[1:1 + d])
    if name == "genz_prodpeak":
        return genz_prodpeak(lo, hi, p[:d], p[d:2 * d])
    if name == "genz_gauss":
        return genz_gauss(lo, hi, p[:d], p[d:2 * d])
    if name == "genz_corner":
        return genz_corner(lo, hi, p[:d])
    raise KeyError(name)
