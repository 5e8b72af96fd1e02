"""Exact arithmetic helpers for the tests (independent of both the oracle and
the CUDA path): k-limb values collapsed to exact integers or Fractions, the
normwise error measure, and a Fraction evaluator of the polynomial, its gradient
and its vector-Jacobian product for tiny cases.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

# normwise relative tolerance per number of limbs k
TOL = {1: 1e-13, 2: 1e-29, 3: 1e-44, 4: 1e-60, 5: 1e-76, 8: 1e-123, 10: 1e-150}


def to_fraction(limbs) -> Fraction:
    return sum((Fraction(float(x)) for x in limbs), Fraction(0))


def series_fractions(a):
    """(k, ..., S) float array -> nested lists of Fractions over the trailing axes."""
    a = np.asarray(a, dtype=np.float64)
    k = a.shape[0]
    flat = a.reshape(k, -1)
    vals = [to_fraction(flat[:, i]) for i in range(flat.shape[1])]
    return np.array(vals, dtype=object).reshape(a.shape[1:])


def exact_ints(arrs):
    """Collapse several (k, ...) float arrays to exact Python ints at one common
    binary scale.  Returns (list of object arrays of ints, scale exponent)."""
    mants, exps = [], []
    for a in arrs:
        a = np.asarray(a, dtype=np.float64)
        m, e = np.frexp(a)
        mi = np.ldexp(m, 53).astype(np.int64)
        ex = e.astype(np.int64) - 53
        mants.append(mi)
        exps.append(ex)
    emin = None
    for mi, ex in zip(mants, exps):
        nz = mi != 0
        if nz.any():
            v = int(ex[nz].min())
            emin = v if emin is None else min(emin, v)
    if emin is None:
        emin = 0
    outs = []
    for mi, ex in zip(mants, exps):
        k = mi.shape[0]
        fm = mi.reshape(k, -1)
        fe = ex.reshape(k, -1)
        vals = np.empty(fm.shape[1], dtype=object)
        for i in range(fm.shape[1]):
            v = 0
            for l in range(k):
                mm = int(fm[l, i])
                if mm:
                    v += mm << (int(fe[l, i]) - emin)
            vals[i] = v
        outs.append(vals.reshape(mi.shape[1:]))
    return outs, emin


def normwise_err(s, r) -> float:
    """max over series of max_j |s_j - r_j| / max_j |r_j|, exact.

    s, r: (k, ..., S) arrays (limb-major), the last axis indexing coefficients.
    A series whose reference is identically zero must be exactly zero (error
    0.0), else the error is reported as inf.
    """
    (si, ri), _ = exact_ints([s, r])
    si = si.reshape(-1, si.shape[-1]) if si.ndim > 1 else si.reshape(1, -1)
    ri = ri.reshape(-1, ri.shape[-1]) if ri.ndim > 1 else ri.reshape(1, -1)
    worst = 0.0
    for a, b in zip(si, ri):
        num = max(abs(int(x) - int(y)) for x, y in zip(a, b))
        den = max(abs(int(y)) for y in b)
        if den == 0:
            err = 0.0 if num == 0 else float("inf")
        else:
            err = num / den
        worst = max(worst, err)
    return worst


def normwise_err_fr(s, ref_fr) -> float:
    """Like normwise_err but against exact Fractions ref_fr (shape (..., S))."""
    sf = series_fractions(s)
    sf = sf.reshape(-1, sf.shape[-1])
    rf = np.asarray(ref_fr, dtype=object).reshape(-1, sf.shape[-1])
    worst = 0.0
    for a, b in zip(sf, rf):
        num = max(abs(x - y) for x, y in zip(a, b))
        den = max(abs(y) for y in b)
        if den == 0:
            err = 0.0 if num == 0 else float("inf")
        else:
            err = float(num / den)
        worst = max(worst, err)
    return worst


# ---------------------------------------------------------------------------
# closed forms for exp-series inputs
# ---------------------------------------------------------------------------

def closed_form_value(supports, coeff_scalars, avals, d: int):
    """Exact value series of c_0 + sum_m c_m exp((sum_{i in S_m} a_i) t), truncated
    at degree d: with inputs z_i = exp(a_i t) and degree-0 coefficients c_m, the
    monomial over S_m is exp((sum_{i in S_m} a_i) t), whose coefficient j is
    (sum a_i)^j / j!.

    coeff_scalars: list of Fractions c_0..c_N.
    """
    out = [Fraction(0)] * (d + 1)
    out[0] += coeff_scalars[0]
    for m, s in enumerate(supports):
        sm = sum(Fraction(avals[i]) for i in s)
        term = Fraction(1)
        for j in range(d + 1):
            out[j] += coeff_scalars[m + 1] * term
            term = term * sm / (j + 1)
    return out


def exp_series_fixed(c: Fraction, P: int, e: int, d: int, F: int):
    """Coefficients 0..d of c exp(sigma t), sigma = P / 2^e, as integers at scale
    2^F: T_0 = c 2^F (exact: c's denominator must divide 2^F) and
    T_j = floor(T_{j-1} P / (2^e j)).  Every floor loses less than one unit and
    a lost unit is carried on multiplied by at most |sigma| / j, so no term is
    off by more than exp(|sigma|) units of 2^-F."""
    num = c.numerator << F
    assert num % c.denominator == 0, "c 2^F is not an integer"
    t = num // c.denominator
    out = [t]
    for j in range(1, d + 1):
        q = t * P
        den = j << e
        t = q // den if q >= 0 else -((-q) // den)  # truncate toward zero: same bound
        out.append(t)
    return out


def limbs_fixed(a, F: int):
    """(k, ..., S) limb array -> object array (..., S) of exact integers at
    scale 2^F (the sum of each coefficient's limbs times 2^F)."""
    a = np.asarray(a, dtype=np.float64)
    k = a.shape[0]
    flat = a.reshape(k, -1)
    out = np.empty(flat.shape[1], dtype=object)
    for i in range(flat.shape[1]):
        v = 0
        for l in range(k):
            x = float(flat[l, i])
            if x != 0.0:
                n_, d_ = x.as_integer_ratio()
                n_ <<= F
                assert n_ % d_ == 0, "limb below 2^-F"
                v += n_ // d_
        out[i] = v
    return out.reshape(a.shape[1:])


def normwise_err_ints(got, ref) -> float:
    """max_j |got_j - ref_j| / max_j |ref_j| of two integer series at one scale."""
    den = max(abs(int(r)) for r in ref)
    num = max(abs(int(g) - int(r)) for g, r in zip(got, ref))
    if den == 0:
        return 0.0 if num == 0 else float("inf")
    return num / den


# ---------------------------------------------------------------------------
# Fraction evaluator (tiny cases only)
# ---------------------------------------------------------------------------

def conv_fr(x, y):
    d = len(x) - 1
    return [sum((x[i] * y[j - i] for i in range(j + 1)), Fraction(0)) for j in range(d + 1)]


def corr_fr(u, s):
    d = len(u) - 1
    return [sum((u[l] * s[l - j] for l in range(j, d + 1)), Fraction(0)) for j in range(d + 1)]


def eval_grad_fr(supports, n, coeff_fr, input_fr):
    """coeff_fr: (N+1, S) Fractions, input_fr: (n, S) Fractions."""
    S = len(coeff_fr[0])
    value = list(coeff_fr[0])
    grad = [[Fraction(0)] * S for _ in range(n)]
    for m, supp in enumerate(supports):
        t = list(coeff_fr[m + 1])
        for v in supp:
            t = conv_fr(t, input_fr[v])
        value = [a + b for a, b in zip(value, t)]
        for i in supp:
            g = list(coeff_fr[m + 1])
            for v in supp:
                if v != i:
                    g = conv_fr(g, input_fr[v])
            grad[i] = [a + b for a, b in zip(grad[i], g)]
    return value, grad


def eval_grad_pow_fr(supports, exponents, n, coeff_fr, input_fr):
    """Monomials with exponents: a_m prod z_v^{e_v}; the partial for x_i is
    e_i a_m z_i^{e_i - 1} prod_{v != i} z_v^{e_v}."""
    S = len(coeff_fr[0])
    value = list(coeff_fr[0])
    grad = [[Fraction(0)] * S for _ in range(n)]

    def power_product(start, supp, ex, skip):
        t = list(start)
        for v, e in zip(supp, ex):
            for _ in range(e - (1 if v == skip else 0)):
                t = conv_fr(t, input_fr[v])
        return t

    for m, (supp, ex) in enumerate(zip(supports, exponents)):
        t = power_product(coeff_fr[m + 1], supp, ex, None)
        value = [a + b for a, b in zip(value, t)]
        for i, e in zip(supp, ex):
            g = power_product(coeff_fr[m + 1], supp, ex, i)
            grad[i] = [a + e * b for a, b in zip(grad[i], g)]
    return value, grad


def vjp_pow_fr(supports, exponents, n, coeff_fr, input_fr, u_fr):
    _, grad = eval_grad_pow_fr(supports, exponents, n, coeff_fr, input_fr)
    gin = [corr_fr(u_fr, grad[i]) for i in range(n)]
    S = len(u_fr)
    gco = [list(u_fr)]
    for supp, ex in zip(supports, exponents):
        mono = [Fraction(1)] + [Fraction(0)] * (S - 1)
        for v, e in zip(supp, ex):
            for _ in range(e):
                mono = conv_fr(mono, input_fr[v])
        gco.append(corr_fr(u_fr, mono))
    return gin, gco


def vjp_fr(supports, n, coeff_fr, input_fr, u_fr):
    S = len(coeff_fr[0])
    _, grad = eval_grad_fr(supports, n, coeff_fr, input_fr)
    gin = [corr_fr(u_fr, grad[i]) for i in range(n)]
    gco = [list(u_fr)]
    for supp in supports:
        mono = list(input_fr[supp[0]])
        for v in supp[1:]:
            mono = conv_fr(mono, input_fr[v])
        gco.append(corr_fr(u_fr, mono))
    return gin, gco


# ---------------------------------------------------------------------------
# complex series as pairs of Fraction lists (tiny cases only)
# ---------------------------------------------------------------------------

def cconv_fr(x, y):
    """x, y: (re, im) pairs of Fraction lists; the truncated complex product."""
    xr, xi = x
    yr, yi = y
    d = len(xr) - 1
    re = [sum((xr[i] * yr[j - i] - xi[i] * yi[j - i] for i in range(j + 1)), Fraction(0)) for j in range(d + 1)]
    im = [sum((xr[i] * yi[j - i] + xi[i] * yr[j - i] for i in range(j + 1)), Fraction(0)) for j in range(d + 1)]
    return re, im


def eval_grad_complex_fr(supports, exponents, n, coeff_fr, input_fr):
    """coeff_fr[m] / input_fr[v]: (re, im) pairs of Fraction lists."""
    S = len(coeff_fr[0][0])
    zero = [Fraction(0)] * S
    one = ([Fraction(1)] + [Fraction(0)] * (S - 1), list(zero))
    exponents = exponents or [[1] * len(s) for s in supports]
    value = (list(coeff_fr[0][0]), list(coeff_fr[0][1]))
    grad = [(list(zero), list(zero)) for _ in range(n)]

    def power_product(start, supp, ex, skip):
        t = start
        for v, e in zip(supp, ex):
            for _ in range(e - (1 if v == skip else 0)):
                t = cconv_fr(t, input_fr[v])
        return t

    for m, (supp, ex) in enumerate(zip(supports, exponents)):
        t = power_product(coeff_fr[m + 1], supp, ex, None)
        value = ([a + b for a, b in zip(value[0], t[0])], [a + b for a, b in zip(value[1], t[1])])
        for i, e in zip(supp, ex):
            g = power_product(coeff_fr[m + 1], supp, ex, i)
            grad[i] = ([a + e * b for a, b in zip(grad[i][0], g[0])], [a + e * b for a, b in zip(grad[i][1], g[1])])
    return value, grad, one
