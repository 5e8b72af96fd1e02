"""Pins of the oracle's multiple double arithmetic against exact rationals.

The oracle rounds every operation from the exact result (Sec. 1: multiple
double numbers are unevaluated sums of k doubles).  Its error must stay below
2^(1-52k) relative, which is well inside every per-k tolerance.
"""
from fractions import Fraction
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_10881_gb300.synth import KS, random_md
from tests.exact import to_fraction, conv_fr, corr_fr, series_fractions


def rel_ok(got_limbs, exact: Fraction, k: int) -> bool:
    err = abs(to_fraction(got_limbs) - exact)
    bound = Fraction(2) ** (1 - 52 * k) * abs(exact)
    return err <= bound


def faithful_limbs(limbs) -> bool:
    """Each limb at most one ulp of the previous one (k-limb normal form)."""
    for a, b in zip(limbs[:-1], limbs[1:]):
        if a == 0.0:
            if b != 0.0:
                return False
            continue
        if abs(b) > math.ulp(a):
            return False
    return True


@pytest.mark.parametrize("k", KS)
def test_md_add_mul_exact(k):
    rng = np.random.default_rng(100 + k)
    x = random_md(rng, k, (40,))
    y = random_md(rng, k, (40,))
    # spread the exponents so that cancellation and gaps are exercised
    scale = np.ldexp(1.0, rng.integers(-60, 60, size=40))
    y = y * scale
    for i in range(40):
        fx, fy = to_fraction(x[:, i]), to_fraction(y[:, i])
        s = O.md_add(x[:, i], y[:, i])
        p = O.md_mul(x[:, i], y[:, i])
        assert rel_ok(s, fx + fy, k)
        assert rel_ok(p, fx * fy, k)
        assert faithful_limbs(s) and faithful_limbs(p)


@pytest.mark.parametrize("k", KS)
def test_md_special_cases(k):
    rng = np.random.default_rng(7 + k)
    x = random_md(rng, k, (1,))[:, 0]
    one = np.zeros(k)
    one[0] = 1.0
    zero = np.zeros(k)
    assert to_fraction(O.md_add(x, -x)) == 0
    assert to_fraction(O.md_mul(x, zero)) == 0
    assert to_fraction(O.md_mul(x, one)) == to_fraction(x)
    assert to_fraction(O.md_add(x, zero)) == to_fraction(x)
    # near-cancellation keeps k limbs of the exact difference
    tiny = np.zeros(k)
    tiny[0] = 2.0 ** -300
    y = O.md_add(x, tiny)
    diff = O.md_add(y, -x)
    assert rel_ok(diff, to_fraction(y) - to_fraction(x), k)


def test_round_sum_exact():
    rng = np.random.default_rng(3)
    for k in KS:
        vals = rng.standard_normal(50) * np.ldexp(1.0, rng.integers(-400, 400, size=50))
        exact = sum((Fraction(float(v)) for v in vals), Fraction(0))
        got = O.round_sum(vals, k)
        assert rel_ok(got, exact, k)
    # exact small sums round exactly
    assert list(O.round_sum([1.0, 2.0 ** -80, -1.0], 2)) == [2.0 ** -80, 0.0]


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("d", [0, 1, 5])
def test_conv_corr_exact(k, d):
    """Eq. (eqconvform) coefficient by coefficient against exact rationals."""
    rng = np.random.default_rng(1000 * k + d)
    x = random_md(rng, k, (d + 1,))
    y = random_md(rng, k, (d + 1,))
    z = O.conv(x, y)
    r = O.corr(x, y)
    xf, yf = list(series_fractions(x)), list(series_fractions(y))
    zf, rf = conv_fr(xf, yf), corr_fr(xf, yf)
    for j in range(d + 1):
        assert rel_ok(z[:, j], zf[j], k) or zf[j] == to_fraction(z[:, j])
        assert rel_ok(r[:, j], rf[j], k) or rf[j] == to_fraction(r[:, j])


def test_conv_known_values():
    """(1 + t)^2 = 1 + 2t + t^2 and (1 - t)(1 + t + t^2 + ...) = 1 truncated."""
    x = np.array([[1.0, 1.0, 0.0, 0.0]])
    assert list(O.conv(x, x)[0]) == [1.0, 2.0, 1.0, 0.0]
    a = np.array([[1.0, -1.0, 0.0, 0.0, 0.0]])
    g = np.ones((1, 5))
    assert list(O.conv(a, g)[0]) == [1.0, 0.0, 0.0, 0.0, 0.0]
    # correlation: r_j = sum_{l>=j} u_l s_{l-j}; with s = delta_0, r = u
    u = np.array([[3.0, 5.0, 7.0]])
    s = np.array([[1.0, 0.0, 0.0]])
    assert list(O.corr(u, s)[0]) == [3.0, 5.0, 7.0]
    # with u = delta_d, r_j = s_{d-j}
    u = np.array([[0.0, 0.0, 1.0]])
    s = np.array([[2.0, 3.0, 4.0]])
    assert list(O.corr(u, s)[0]) == [4.0, 3.0, 2.0]
