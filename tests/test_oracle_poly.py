"""Pins of the oracle's polynomial evaluation, gradient and VJP.

Each check is independent of the oracle's own arithmetic: exact rationals on
tiny inputs, closed forms for exp-series inputs, float64 at k=1, Euler's
identity for homogeneous polynomials, and exact central differences (every
variable appears with exponent 1, so the value is affine in each input series
and in each coefficient series).
"""
from fractions import Fraction
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_10881_gb300 import synth
from paper_2101_10881_gb300.synth import KS, random_md
from tests.exact import (TOL, closed_form_value, eval_grad_fr, normwise_err, normwise_err_fr, series_fractions,
                         to_fraction, vjp_fr, conv_fr)


def tiny_case(rng, k, n, N, d, lo=1, hi=None):
    hi = hi or n
    supports = synth.random_supports(rng, n, N, lo, hi)
    coeff = random_md(rng, k, (N + 1, d + 1))
    inputs = random_md(rng, k, (n, d + 1))
    return supports, coeff, inputs


@pytest.mark.parametrize("k", KS)
def test_eval_grad_exact_tiny(k):
    rng = np.random.default_rng(50 + k)
    for trial in range(3):
        n = int(rng.integers(1, 7))
        N = int(rng.integers(0, 9))
        d = int(rng.integers(0, 5))
        supports, coeff, inputs = tiny_case(rng, k, n, N, d)
        v, g = O.eval_grad(supports, n, coeff, inputs)
        cf = series_fractions(coeff)
        zf = series_fractions(inputs)
        vf, gf = eval_grad_fr(supports, n, cf, zf)
        assert normwise_err_fr(v, [vf]) <= TOL[k]
        assert normwise_err_fr(g, gf) <= TOL[k]


def test_paper_example_polynomial():
    """p = a0 + a1 x1 x3 x6 + a2 x1 x2 x5 x6 + a3 x2 x3 x4 (Eq. eqexpoly): the
    six partials listed after Eq. (eqparallel), read with the index fixes
    b_{2,2} and c_{3,1}."""
    k, d, n = 2, 3, 6
    supports = [[0, 2, 5], [0, 1, 4, 5], [1, 2, 3]]
    rng = np.random.default_rng(11)
    coeff = random_md(rng, k, (4, d + 1))
    inputs = random_md(rng, k, (n, d + 1))
    v, g = O.eval_grad(supports, n, coeff, inputs)
    a = series_fractions(coeff)
    z = series_fractions(inputs)
    C = conv_fr

    def prod(*s):
        out = s[0]
        for t in s[1:]:
            out = C(out, t)
        return out

    def add(*s):
        return [sum(c, Fraction(0)) for c in zip(*s)]

    expect = [
        add(prod(a[1], z[2], z[5]), prod(a[2], z[1], z[4], z[5])),   # b11 + b22
        add(prod(a[2], z[0], z[4], z[5]), prod(a[3], z[2], z[3])),   # c21 + b31
        add(prod(a[1], z[0], z[5]), prod(a[3], z[1], z[3])),         # c11 + c31
        prod(a[3], z[1], z[2]),                                      # f32
        prod(a[2], z[0], z[1], z[5]),                                # c22
        add(prod(a[1], z[0], z[2]), prod(a[2], z[0], z[1], z[4])),   # f12 + f23
    ]
    assert normwise_err_fr(g, expect) <= TOL[k]
    value = add(a[0], prod(a[1], z[0], z[2], z[5]), prod(a[2], z[0], z[1], z[4], z[5]),
                prod(a[3], z[1], z[2], z[3]))
    assert normwise_err_fr(v, [value]) <= TOL[k]


@pytest.mark.parametrize("k", [1, 2, 4, 8, 10])
def test_closed_form_exp_inputs(k):
    """z_i = exp(a_i t): the monomial over S equals exp((sum_S a_i) t) and its
    partial w.r.t. x_i equals exp((sum_S a_i - a_i) t) (Sec. 8 pin 2)."""
    d, n, N = 12, 8, 10
    rng = np.random.default_rng(200 + k)
    avals = [float(a) for a in rng.uniform(-1, 1, size=n)]
    inputs = synth.exp_inputs(avals, d, k)
    supports = synth.random_supports(rng, n, N, 2, 5)
    coeff = synth.scalar_coeffs(rng, k, N, d)
    cs = [to_fraction(coeff[:, m, 0]) for m in range(N + 1)]
    v, g = O.eval_grad(supports, n, coeff, inputs)
    vexact = closed_form_value(supports, cs, avals, d)
    assert normwise_err_fr(v, [vexact]) <= TOL[k]
    gexact = []
    for i in range(n):
        gi = [Fraction(0)] * (d + 1)
        for m, s in enumerate(supports):
            if i not in s:
                continue
            sm = sum(Fraction(avals[v_]) for v_ in s if v_ != i)
            term = Fraction(1)
            for j in range(d + 1):
                gi[j] += cs[m + 1] * term
                term = term * sm / (j + 1)
        gexact.append(gi)
    assert normwise_err_fr(g, gexact) <= TOL[k]


def test_k1_matches_float64():
    """At k=1 the oracle agrees with a plain float64 evaluation (numpy)."""
    rng = np.random.default_rng(5)
    n, N, d = 7, 20, 9
    supports = synth.random_supports(rng, n, N, 1, 5)
    coeff = rng.uniform(-1, 1, size=(1, N + 1, d + 1))
    inputs = rng.uniform(-1, 1, size=(1, n, d + 1))
    v, g = O.eval_grad(supports, n, coeff, inputs)

    def cv(x, y):
        return np.convolve(x, y)[: d + 1]

    vv = coeff[0, 0].copy()
    gg = np.zeros((n, d + 1))
    for m, s in enumerate(supports):
        t = coeff[0, m + 1]
        for x in s:
            t = cv(t, inputs[0, x])
        vv += t
        for i in s:
            t = coeff[0, m + 1]
            for x in s:
                if x != i:
                    t = cv(t, inputs[0, x])
            gg[i] += t
    assert np.max(np.abs(v[0] - vv)) / np.max(np.abs(vv)) < 1e-13
    for i in range(n):
        den = np.max(np.abs(gg[i]))
        if den == 0:
            assert np.all(g[0, i] == 0)
        else:
            assert np.max(np.abs(g[0, i] - gg[i])) / den < 1e-13


def test_d0_is_scalar_arithmetic():
    rng = np.random.default_rng(8)
    k, n, N = 3, 5, 6
    supports = synth.random_supports(rng, n, N, 1, 4)
    coeff = random_md(rng, k, (N + 1, 1))
    inputs = random_md(rng, k, (n, 1))
    v, g = O.eval_grad(supports, n, coeff, inputs)
    a = [to_fraction(coeff[:, m, 0]) for m in range(N + 1)]
    z = [to_fraction(inputs[:, i, 0]) for i in range(n)]
    val = a[0] + sum(a[m + 1] * math.prod(z[i] for i in s) for m, s in enumerate(supports))
    assert abs(to_fraction(v[:, 0]) - val) <= abs(val) * Fraction(2) ** (-150)
    for i in range(n):
        gi = sum(a[m + 1] * math.prod(z[j] for j in s if j != i)
                 for m, s in enumerate(supports) if i in s)
        assert abs(to_fraction(g[:, i, 0]) - gi) <= abs(gi) * Fraction(2) ** (-150) + Fraction(0)


@pytest.mark.parametrize("k", [2, 4])
def test_euler_identity_homogeneous(k):
    """p1-like polynomial, homogeneous of degree m: sum_i z_i * g_i = m (v - a_0)."""
    n, m, d = 7, 3, 6
    supports = synth.supports_p1(n, m)
    prob = synth.make_problem("euler", supports, n, d, k, seed=9)
    v, g = O.eval_grad(supports, n, prob.coeff, prob.inputs)
    zf = series_fractions(prob.inputs)
    gf = series_fractions(g)
    lhs = [Fraction(0)] * (d + 1)
    for i in range(n):
        lhs = [a + b for a, b in zip(lhs, conv_fr(list(zf[i]), list(gf[i])))]
    vf = series_fractions(v)
    a0 = series_fractions(prob.coeff[:, 0])
    rhs = [m * (x - y) for x, y in zip(vf, a0)]
    num = max(abs(x - y) for x, y in zip(lhs, rhs))
    den = max(abs(y) for y in rhs)
    assert float(num / den) <= 50 * TOL[k]


def test_gradient_is_central_difference_of_value():
    """The value is affine in each input coefficient z_i[j]: a central difference
    of the value reproduces the gradient series shifted by j."""
    k, n, N, d = 8, 5, 9, 6
    rng = np.random.default_rng(12)
    supports, coeff, inputs = tiny_case(rng, k, n, N, d)
    _, g = O.eval_grad(supports, n, coeff, inputs)
    h = 2.0 ** -20
    for trial in range(6):
        i = int(rng.integers(0, n))
        j = int(rng.integers(0, d + 1))
        zp, zm = inputs.copy(), inputs.copy()
        zp[0, i, j] += h
        zm[0, i, j] -= h
        vp = series_fractions(O.eval_grad(supports, n, coeff, zp, grad=False))
        vm = series_fractions(O.eval_grad(supports, n, coeff, zm, grad=False))
        gi = series_fractions(g[:, i])
        fd = [(a - b) / (2 * Fraction(h)) for a, b in zip(vp, vm)]
        expect = [Fraction(0)] * j + list(gi[: d + 1 - j])
        num = max(abs(a - b) for a, b in zip(fd, expect))
        den = max(max(abs(b) for b in gi), Fraction(1, 10 ** 30))
        assert float(num / den) < 1e-90


@pytest.mark.parametrize("k", [1, 3, 10])
def test_vjp_exact_tiny(k):
    rng = np.random.default_rng(70 + k)
    for trial in range(2):
        n = int(rng.integers(1, 6))
        N = int(rng.integers(1, 7))
        d = int(rng.integers(0, 5))
        supports, coeff, inputs = tiny_case(rng, k, n, N, d)
        u = random_md(rng, k, (d + 1,))
        gi, gc = O.vjp(supports, n, coeff, inputs, u)
        gif, gcf = vjp_fr(supports, n, series_fractions(coeff), series_fractions(inputs),
                          list(series_fractions(u)))
        assert normwise_err_fr(gi, gif) <= TOL[k]
        assert normwise_err_fr(gc, gcf) <= TOL[k]


def test_vjp_central_difference_coefficients():
    """L = <u, v> is affine in each coefficient series a_m, so a central
    difference along a direction inside a_m is exact up to rounding."""
    k, n, N, d = 8, 4, 6, 5
    rng = np.random.default_rng(21)
    supports, coeff, inputs = tiny_case(rng, k, n, N, d)
    u = random_md(rng, k, (d + 1,))
    _, gc = O.vjp(supports, n, coeff, inputs, u)
    uf = series_fractions(u)
    h = 2.0 ** -20
    for m in range(N + 1):
        dirn = np.ldexp(rng.integers(-8, 9, size=d + 1).astype(float), -3)
        cp, cm = coeff.copy(), coeff.copy()
        cp[0, m] += h * dirn
        cm[0, m] -= h * dirn
        vp = series_fractions(O.eval_grad(supports, n, cp, inputs, grad=False))
        vm = series_fractions(O.eval_grad(supports, n, cm, inputs, grad=False))
        Lp = sum(a * b for a, b in zip(uf, vp))
        Lm = sum(a * b for a, b in zip(uf, vm))
        fd = (Lp - Lm) / (2 * Fraction(h))
        an = sum(to_fraction(gc[:, m, j]) * Fraction(float(dirn[j])) for j in range(d + 1))
        scale = max(abs(an), Fraction(1, 10 ** 6))
        assert float(abs(fd - an) / scale) < 1e-90


def test_oracle_thread_count_invariance():
    """Exact accumulation makes the result independent of the thread count."""
    rng = np.random.default_rng(31)
    supports, coeff, inputs = tiny_case(rng, 4, 6, 30, 7, lo=1, hi=4)
    v1, g1 = O.eval_grad(supports, 6, coeff, inputs, nthreads=1)
    v4, g4 = O.eval_grad(supports, 6, coeff, inputs, nthreads=4)
    assert np.array_equal(v1, v4) and np.array_equal(g1, g4)


def test_empty_polynomial_and_unused_variable():
    k, n, d = 2, 4, 3
    rng = np.random.default_rng(2)
    coeff = random_md(rng, k, (1, d + 1))
    inputs = random_md(rng, k, (n, d + 1))
    v, g = O.eval_grad([], n, coeff, inputs)
    assert np.array_equal(v, coeff[:, 0])
    assert np.all(g == 0)
    coeff2 = random_md(rng, k, (2, d + 1))
    v, g = O.eval_grad([[1]], n, coeff2, inputs)
    # x_1 alone: gradient of a_1 x_1 is a_1, other partials vanish
    assert np.array_equal(g[:, 1], coeff2[:, 1])
    assert np.all(g[:, 0] == 0) and np.all(g[:, 2] == 0) and np.all(g[:, 3] == 0)


def test_invalid_supports_rejected():
    k, n, d = 1, 3, 2
    coeff = np.zeros((k, 2, d + 1))
    inputs = np.zeros((k, n, d + 1))
    for bad in ([[2, 1]], [[0, 0]], [[3]], [[-1]], [[]]):
        with pytest.raises(ValueError):
            O.eval_grad(bad, n, coeff, inputs)
