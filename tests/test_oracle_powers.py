"""Pins of the oracle for monomials with positive powers (Sec. 3: a monomial
x_1^3 x_2^5 is the common factor x_1^2 x_2^4 times x_1 x_2).

The oracle forms every power by repeated multiplication and every partial
derivative e_i a z_i^(e_i - 1) prod_(v != i) z_v^(e_v) afresh, adding it e_i
times.  It is checked against exact rationals on tiny inputs, the closed forms
of exp-series inputs (a product of powers of exp(a_i t) is exp((sum e_i a_i) t)),
the same polynomial written with repeated variables, and exact central
differences (with exponents at most 2 the value is quadratic in each input
coefficient).
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_10881_gb300 import synth
from paper_2101_10881_gb300.synth import KS, random_md
from tests.exact import (TOL, eval_grad_pow_fr, normwise_err, normwise_err_fr, series_fractions,
                         to_fraction, vjp_pow_fr)


def random_exponents(rng, supports, hi):
    return [[int(e) for e in rng.integers(1, hi + 1, size=len(s))] for s in supports]


@pytest.mark.parametrize("k", KS)
def test_powers_exact_tiny(k):
    rng = np.random.default_rng(700 + k)
    for trial in range(3):
        n = int(rng.integers(1, 5))
        N = int(rng.integers(1, 6))
        d = int(rng.integers(0, 5))
        supp = synth.random_supports(rng, n, N, 1, n)
        ex = random_exponents(rng, supp, 3)
        coeff = random_md(rng, k, (N + 1, d + 1))
        inputs = random_md(rng, k, (n, d + 1))
        v, g = O.eval_grad(supp, n, coeff, inputs, exponents=ex)
        vf, gf = eval_grad_pow_fr(supp, ex, n, series_fractions(coeff), series_fractions(inputs))
        assert normwise_err_fr(v, [vf]) <= TOL[k]
        assert normwise_err_fr(g, gf) <= TOL[k]


@pytest.mark.parametrize("k", [2, 10])
def test_powers_closed_form_exp_inputs(k):
    """z_i = exp(a_i t): prod z_i^{e_i} = exp(s t) with s = sum e_i a_i, and the
    partial for x_i is e_i exp((s - a_i) t)."""
    d, n, N = 16, 6, 8
    rng = np.random.default_rng(710 + k)
    avals = [float(a) for a in rng.uniform(-1, 1, size=n)]
    inputs = synth.exp_inputs(avals, d, k)
    supp = synth.random_supports(rng, n, N, 1, 4)
    ex = random_exponents(rng, supp, 4)
    coeff = synth.scalar_coeffs(rng, k, N, d)
    cs = [to_fraction(coeff[:, m, 0]) for m in range(N + 1)]
    v, g = O.eval_grad(supp, n, coeff, inputs, exponents=ex)

    def exp_series(rate, scale):
        out, term = [], Fraction(scale)
        for j in range(d + 1):
            out.append(term)
            term = term * rate / (j + 1)
        return out

    vexact = [cs[0] if j == 0 else Fraction(0) for j in range(d + 1)]
    gexact = [[Fraction(0)] * (d + 1) for _ in range(n)]
    for m, (s, e) in enumerate(zip(supp, ex)):
        rate = sum(Fraction(avals[i]) * ei for i, ei in zip(s, e))
        vexact = [a + b for a, b in zip(vexact, exp_series(rate, cs[m + 1]))]
        for i, ei in zip(s, e):
            gexact[i] = [a + b for a, b in zip(gexact[i], exp_series(rate - Fraction(avals[i]), cs[m + 1] * ei))]
    assert normwise_err_fr(v, [vexact]) <= TOL[k]
    assert normwise_err_fr(g, gexact) <= TOL[k]


def test_powers_as_repeated_variables():
    """x0^2 x1^3 written as x0 x2 x1 x3 x4 with z2 = z0 and z3 = z4 = z1: the
    same value, and the partial for x0 (x1) is the sum of the partials for its
    copies."""
    k, d = 4, 9
    rng = np.random.default_rng(720)
    z = random_md(rng, k, (2, d + 1))
    coeff = random_md(rng, k, (2, d + 1))
    v, g = O.eval_grad([[0, 1]], 2, coeff, z, exponents=[[2, 3]])
    zd = np.stack([z[:, 0], z[:, 1], z[:, 0], z[:, 1], z[:, 1]], axis=1)
    vd, gd = O.eval_grad([[0, 1, 2, 3, 4]], 5, coeff, zd)
    assert normwise_err(v, vd) <= TOL[k]
    gdf = series_fractions(gd)
    gf = series_fractions(g)
    for j in range(d + 1):
        for mine, copies in ((gf[0][j], gdf[0][j] + gdf[2][j]), (gf[1][j], gdf[1][j] + gdf[3][j] + gdf[4][j])):
            assert abs(mine - copies) <= abs(copies) * Fraction(TOL[k]) + Fraction(1, 10 ** 300)


def test_exponents_one_equal_plain_call():
    k, d, n = 3, 7, 6
    rng = np.random.default_rng(730)
    supp = synth.random_supports(rng, n, 7, 1, 5)
    coeff = random_md(rng, k, (len(supp) + 1, d + 1))
    inputs = random_md(rng, k, (n, d + 1))
    v, g = O.eval_grad(supp, n, coeff, inputs)
    v1, g1 = O.eval_grad(supp, n, coeff, inputs, exponents=[[1] * len(s) for s in supp])
    assert np.array_equal(v, v1) and np.array_equal(g, g1)


@pytest.mark.parametrize("k", [2, 4])
def test_vjp_powers_exact_tiny(k):
    rng = np.random.default_rng(740 + k)
    n, N, d = 3, 4, 4
    supp = synth.random_supports(rng, n, N, 1, 3)
    ex = random_exponents(rng, supp, 3)
    coeff = random_md(rng, k, (N + 1, d + 1))
    inputs = random_md(rng, k, (n, d + 1))
    u = random_md(rng, k, (d + 1,))
    gi, gc = O.vjp(supp, n, coeff, inputs, u, exponents=ex)
    fi, fc = vjp_pow_fr(supp, ex, n, series_fractions(coeff), series_fractions(inputs), series_fractions(u))
    assert normwise_err_fr(gi, fi) <= TOL[k]
    assert normwise_err_fr(gc, fc) <= TOL[k]


def test_vjp_powers_central_differences():
    """With exponents at most 2, L = <u, v> is a polynomial of degree at most 2
    in any one input coefficient, so the central difference along it is exact
    (up to the rounding of L itself, far below the octo double tolerance)."""
    k, d, n = 8, 6, 4
    rng = np.random.default_rng(750)
    supp = [[0, 1], [1, 2, 3], [0, 3]]
    ex = [[2, 1], [1, 2, 2], [2, 2]]
    coeff = random_md(rng, k, (len(supp) + 1, d + 1))
    inputs = random_md(rng, k, (n, d + 1))
    u = random_md(rng, k, (d + 1,))
    gi, _ = O.vjp(supp, n, coeff, inputs, u, exponents=ex)
    uf = series_fractions(u)

    def L(z):
        v = O.eval_grad(supp, n, coeff, z, grad=False, exponents=ex)
        vf = series_fractions(v)
        return sum(a * b for a, b in zip(uf, vf))

    h = 2.0 ** -20
    gif = series_fractions(gi)
    for _ in range(6):
        i, j = int(rng.integers(0, n)), int(rng.integers(0, d + 1))
        zp, zm = inputs.copy(), inputs.copy()
        zp[:, i, j] = 0.0
        zm[:, i, j] = 0.0
        base = to_fraction(inputs[:, i, j])
        zp[:, i, j] = synth.round_fraction_to_limbs(base + Fraction(h), k)
        zm[:, i, j] = synth.round_fraction_to_limbs(base - Fraction(h), k)
        fd = (L(zp) - L(zm)) / (2 * Fraction(h))
        ref = gif[i][j]
        scale = max(abs(x) for x in gif.ravel())
        assert abs(fd - ref) <= scale * Fraction(TOL[k])


def test_invalid_exponents_rejected():
    k, d = 2, 3
    coeff = np.zeros((k, 2, d + 1))
    z = np.zeros((k, 2, d + 1))
    for bad in ([[0, 1]], [[1, -2]], [[65, 1]]):
        with pytest.raises(Exception):
            O.eval_grad([[0, 1]], 2, coeff, z, exponents=bad)
