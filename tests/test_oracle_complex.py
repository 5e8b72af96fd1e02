"""Pins of the oracle for complex coefficient and input series (the complex
variant of the method: real and imaginary parts as separate k-double series,
a complex product as four real ones).

Checked against exact complex rationals on tiny inputs, the closed forms of
exp-series inputs with complex rates, the real oracle when every imaginary
part is zero (bit for bit), and conjugation (conjugate coefficients and inputs
give the conjugate results, bit for bit).  The VJP over complex series (real
and imaginary parts as real variables) against exact central differences of
the real loss, the real VJP at zero imaginary parts, conjugation and rotation
of the upstream series by i."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_10881_gb300 import synth
from paper_2101_10881_gb300.synth import KS, random_md
from tests.exact import TOL, eval_grad_complex_fr, normwise_err_fr, series_fractions, to_fraction


def complex_case(rng, k, n, N, d):
    supp = synth.random_supports(rng, n, N, 1, n)
    coeff = np.stack([random_md(rng, k, (N + 1, d + 1)), random_md(rng, k, (N + 1, d + 1))])
    inputs = np.stack([random_md(rng, k, (n, d + 1)), random_md(rng, k, (n, d + 1))])
    return supp, coeff, inputs


def pairs(a):
    """(2, k, series, S) -> per series a (re, im) pair of Fraction lists."""
    re, im = series_fractions(a[0]), series_fractions(a[1])
    return [(list(re[t]), list(im[t])) for t in range(re.shape[0])]


@pytest.mark.parametrize("k", KS)
def test_complex_exact_tiny(k):
    rng = np.random.default_rng(1100 + k)
    for _ in range(2):
        n = int(rng.integers(1, 4))
        N = int(rng.integers(1, 5))
        d = int(rng.integers(0, 4))
        supp, coeff, inputs = complex_case(rng, k, n, N, d)
        ex = [[int(e) for e in rng.integers(1, 3, size=len(s))] for s in supp]
        v, g = O.eval_grad_complex(supp, n, coeff, inputs, exponents=ex)
        vf, gf, _ = eval_grad_complex_fr(supp, ex, n, pairs(coeff), pairs(inputs))
        assert normwise_err_fr(v[0], [vf[0]]) <= TOL[k] and normwise_err_fr(v[1], [vf[1]]) <= TOL[k]
        assert normwise_err_fr(g[0], [gi[0] for gi in gf]) <= TOL[k]
        assert normwise_err_fr(g[1], [gi[1] for gi in gf]) <= TOL[k]


def test_complex_with_zero_imaginary_parts_is_the_real_oracle():
    k, d, n = 4, 10, 5
    rng = np.random.default_rng(1110)
    supp = synth.random_supports(rng, n, 7, 1, 4)
    coeff = random_md(rng, k, (len(supp) + 1, d + 1))
    inputs = random_md(rng, k, (n, d + 1))
    v, g = O.eval_grad(supp, n, coeff, inputs)
    cv, cg = O.eval_grad_complex(supp, n, np.stack([coeff, 0 * coeff]), np.stack([inputs, 0 * inputs]))
    assert np.array_equal(cv[0], v) and np.array_equal(cg[0], g)
    assert not cv[1].any() and not cg[1].any()


def test_complex_conjugation():
    k, d, n = 3, 8, 4
    rng = np.random.default_rng(1120)
    supp, coeff, inputs = complex_case(rng, k, n, 6, d)
    v, g = O.eval_grad_complex(supp, n, coeff, inputs)
    cc = coeff.copy()
    cc[1] = -cc[1]
    ci = inputs.copy()
    ci[1] = -ci[1]
    w, h = O.eval_grad_complex(supp, n, cc, ci)
    assert np.array_equal(w[0], v[0]) and np.array_equal(w[1], -v[1])
    assert np.array_equal(h[0], g[0]) and np.array_equal(h[1], -g[1])


@pytest.mark.parametrize("k", [2, 8])
def test_complex_closed_form_exp_inputs(k):
    """z_v = exp(a_v t) with complex a_v: prod z_v^{e_v} = exp(s t),
    s = sum e_v a_v; coefficient j is s^j / j! (complex rationals)."""
    d, n = 12, 4
    rng = np.random.default_rng(1130 + k)
    a = [(Fraction(float(x)), Fraction(float(y))) for x, y in rng.uniform(-1, 1, size=(n, 2))]

    def cmul(p, q):
        return (p[0] * q[0] - p[1] * q[1], p[0] * q[1] + p[1] * q[0])

    def exp_coeffs(rate, scale):
        out, term = [], scale
        for j in range(d + 1):
            out.append(term)
            term = cmul(term, rate)
            term = (term[0] / (j + 1), term[1] / (j + 1))
        return out

    inputs = np.zeros((2, k, n, d + 1))
    for v in range(n):
        for j, c in enumerate(exp_coeffs(a[v], (Fraction(1), Fraction(0)))):
            inputs[0, :, v, j] = synth.round_fraction_to_limbs(c[0], k)
            inputs[1, :, v, j] = synth.round_fraction_to_limbs(c[1], k)
    supp = [[0, 1], [1, 2, 3], [0, 3], [2]]
    ex = [[2, 1], [1, 1, 3], [1, 2], [3]]
    N = len(supp)
    coeff = np.zeros((2, k, N + 1, d + 1))
    coeff[:, :, :, 0] = np.stack([random_md(rng, k, (N + 1,)), random_md(rng, k, (N + 1,))])
    cs = [(to_fraction(coeff[0, :, m, 0]), to_fraction(coeff[1, :, m, 0])) for m in range(N + 1)]
    v, _ = O.eval_grad_complex(supp, n, coeff, inputs, exponents=ex)
    want_re = [cs[0][0]] + [Fraction(0)] * d
    want_im = [cs[0][1]] + [Fraction(0)] * d
    for m, (s_, e_) in enumerate(zip(supp, ex)):
        rate = (sum(a[v][0] * e for v, e in zip(s_, e_)), sum(a[v][1] * e for v, e in zip(s_, e_)))
        for j, c in enumerate(exp_coeffs(rate, cs[m + 1])):
            want_re[j] += c[0]
            want_im[j] += c[1]
    # rounding the inputs to k limbs perturbs the value far below the tolerance
    assert normwise_err_fr(v[0], [want_re]) <= TOL[k]
    assert normwise_err_fr(v[1], [want_im]) <= TOL[k]


# ---------------------------------------------------------------------------
# VJP over complex series (real and imaginary parts as real variables)
# ---------------------------------------------------------------------------

def loss_fr(supp, n, cp, ip, up):
    """L = sum_j Re u_j Re v_j + Im u_j Im v_j, exactly (exponents one)."""
    vf, _, _ = eval_grad_complex_fr(supp, None, n, cp, ip)
    return sum(a * b for a, b in zip(up[0], vf[0])) + sum(a * b for a, b in zip(up[1], vf[1]))


@pytest.mark.parametrize("k", [1, 2, 4, 10])
def test_complex_vjp_central_differences_exact(k):
    """With exponents one the value is affine in every real and imaginary part
    of every input coefficient and coefficient-series coefficient, so the
    central difference (L(x + h) - L(x - h)) / 2h of the exact loss is the exact
    derivative: every component of the oracle's gradients (dL/dRe in block 0,
    dL/dIm in block 1) against it.  Independent of how the oracle forms the
    gradient (no conjugate correlation here)."""
    rng = np.random.default_rng(1200 + k)
    n, N, d = 3, 3, 3
    supp, coeff, inputs = complex_case(rng, k, n, N, d)
    u = np.stack([random_md(rng, k, (d + 1,)), random_md(rng, k, (d + 1,))])
    gi, gc = O.vjp_complex(supp, n, coeff, inputs, u)
    cp, ip = pairs(coeff), pairs(inputs)
    up = (list(series_fractions(u[0])), list(series_fractions(u[1])))
    h = Fraction(1, 1 << 20)
    for which, base, grad in (("input", ip, gi), ("coeff", cp, gc)):
        for s_ in range(len(base)):
            for part in (0, 1):
                exact = []
                for j in range(d + 1):
                    lo = [(list(a), list(b)) for a, b in base]
                    hi = [(list(a), list(b)) for a, b in base]
                    lo[s_][part][j] -= h
                    hi[s_][part][j] += h
                    if which == "input":
                        fd = (loss_fr(supp, n, cp, hi, up) - loss_fr(supp, n, cp, lo, up)) / (2 * h)
                    else:
                        fd = (loss_fr(supp, n, hi, ip, up) - loss_fr(supp, n, lo, ip, up)) / (2 * h)
                    exact.append(fd)
                assert normwise_err_fr(grad[part][:, s_], [exact]) <= TOL[k], (which, s_, part)


def test_complex_vjp_with_zero_imaginary_parts_is_the_real_vjp():
    k, d, n = 3, 9, 4
    rng = np.random.default_rng(1210)
    supp = synth.random_supports(rng, n, 6, 1, 4)
    coeff = random_md(rng, k, (len(supp) + 1, d + 1))
    inputs = random_md(rng, k, (n, d + 1))
    u = random_md(rng, k, (d + 1,))
    ri, rc = O.vjp(supp, n, coeff, inputs, u)
    gi, gc = O.vjp_complex(supp, n, np.stack([coeff, 0 * coeff]), np.stack([inputs, 0 * inputs]),
                           np.stack([u, 0 * u]))
    assert np.array_equal(gi[0], ri) and np.array_equal(gc[0], rc)
    assert not gi[1].any() and not gc[1].any()


def test_complex_vjp_conjugation_and_rotation():
    """Conjugating coefficients, inputs and upstream conjugates both gradients;
    multiplying the upstream by i multiplies them by i (bit for bit)."""
    k, d, n = 2, 7, 3
    rng = np.random.default_rng(1220)
    supp, coeff, inputs = complex_case(rng, k, n, 5, d)
    u = np.stack([random_md(rng, k, (d + 1,)), random_md(rng, k, (d + 1,))])
    gi, gc = O.vjp_complex(supp, n, coeff, inputs, u)
    conj = lambda a: np.stack([a[0], -a[1]])  # noqa: E731
    hi, hc = O.vjp_complex(supp, n, conj(coeff), conj(inputs), conj(u))
    assert np.array_equal(hi, conj(gi)) and np.array_equal(hc, conj(gc))
    iu = np.stack([-u[1], u[0]])
    ji, jc = O.vjp_complex(supp, n, coeff, inputs, iu)
    assert np.array_equal(ji, np.stack([-gi[1], gi[0]])) and np.array_equal(jc, np.stack([-gc[1], gc[0]]))
