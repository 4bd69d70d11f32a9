"""The Nose-Hoover chain's small-argument exponential (a degree-6 Taylor
polynomial for |x| <= 1/64, exp() beyond): its truncation error is below
half an FP64 ulp of e^x on the whole interval, so the GPU routine differs from
a correctly rounded e^x only by the rounding of its six FMAs.  Checked in
50-digit decimal arithmetic against e^x itself (not against the same
polynomial)."""
from decimal import Decimal, getcontext
from math import factorial

import numpy as np
import pytest


def _trunc_rel_error(x: Decimal) -> Decimal:
    poly = Decimal(1) + sum(x ** n / factorial(n) for n in range(1, 7))
    return abs(poly - x.exp()) / x.exp()


def test_series_truncation_below_half_ulp():
    getcontext().prec = 50
    half_ulp = Decimal(2) ** -53
    xs = [Decimal(v) for v in np.linspace(-1 / 64, 1 / 64, 257)]
    worst = max(_trunc_rel_error(x) for x in xs)
    # the bound of the comment: |x|^7 / 7! e^|x| at the interval's ends
    bound = (Decimal(1) / 64) ** 7 / factorial(7) * (Decimal(1) / 64).exp()
    assert worst <= bound < half_ulp / 2


def test_degree_five_would_not_do():
    # the degree is not larger than needed by much: one term fewer misses
    # half an ulp at the interval's end
    getcontext().prec = 50
    x = Decimal(1) / 64
    poly5 = sum(x ** n / factorial(n) for n in range(6))
    assert abs(poly5 - x.exp()) / x.exp() > Decimal(2) ** -53
