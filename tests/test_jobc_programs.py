"""The job compiler's whole programs (pes_jobc_program) run on the host by an
exact interpreter: every slot a series of exact rationals, every job executed
as written (convolution, correlation, addition, subtraction), every output
summed from the addition tables.  Without any rounding the results must equal
the exact value, gradient and VJP, which pins the tables themselves: the real
reverse mode with powers, the complex form (four real products and the add /
subtract jobs of every complex product, correlations with the conjugate in the
VJP), systems (per-polynomial constants, Jacobian outputs, one upstream series
per polynomial) and the VJP tables.  No GPU needed."""
from fractions import Fraction

import numpy as np
import pytest

from paper_2101_10881_gb300 import pes, synth
from tests.exact import cconv_fr, conv_fr, corr_fr, eval_grad_complex_fr, eval_grad_pow_fr, vjp_pow_fr

CONV, CORR, ADD, SUB = 0, 1, 2, 3


@pytest.fixture(scope="module", autouse=True)
def built():
    pes.build()


def rand_series(rng, S):
    return [Fraction(int(rng.integers(-9, 10)), int(rng.integers(1, 8))) for _ in range(S)]


def run_jobs(slots, jobs):
    for in1, in2, out, _layer, kind in jobs:
        x, y = slots[int(in1)], slots[int(in2)]
        S = len(x)
        if kind == CONV:
            slots[int(out)] = conv_fr(x, y)
        elif kind == CORR:
            slots[int(out)] = [sum((x[j + i] * y[i] for i in range(S - j)), Fraction(0)) for j in range(S)]
        elif kind == ADD:
            slots[int(out)] = [a + b for a, b in zip(x, y)]
        elif kind == SUB:
            slots[int(out)] = [a - b for a, b in zip(x, y)]
        else:
            raise AssertionError(f"unknown job kind {kind}")


def output(P, slots, o, S):
    acc = [Fraction(0)] * S
    for t in range(int(P["add_ptr"][o]), int(P["add_ptr"][o + 1])):
        src, mu = int(P["add_src"][t]), int(P["add_mult"][t])
        acc = [a + mu * b for a, b in zip(acc, slots[src])]
    return acc


def case(seed, powers):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 5))
    supp = synth.random_supports(rng, n, int(rng.integers(1, 5)), 1, n)
    ex = [[int(e) for e in rng.integers(1, 4, size=len(s))] for s in supp] if powers else None
    return rng, n, supp, ex


@pytest.mark.parametrize("powers", [False, True])
@pytest.mark.parametrize("seed", range(4))
def test_real_program_exact(seed, powers):
    rng, n, supp, ex = case(3000 + seed, powers)
    N, S = len(supp), 4
    P = pes.jobc_program(supp, n, exponents=ex, with_vjp=True)
    coeff = [rand_series(rng, S) for _ in range(N + 1)]
    z = [rand_series(rng, S) for _ in range(n)]
    u = rand_series(rng, S)
    exps = ex or [[1] * len(s) for s in supp]
    # evaluation
    slots = {m: coeff[m] for m in range(N + 1)}
    slots.update({1 + N + i: z[i] for i in range(n)})
    assert P["input_slots"] == 1 + N + n
    run_jobs(slots, P["jobs"])
    value, grad = eval_grad_pow_fr(supp, exps, n, coeff, z)
    assert output(P, slots, 0, S) == value
    for i in range(n):
        assert output(P, slots, 1 + i, S) == grad[i]
    # VJP: the forward and monomial products afresh, the gradient series into
    # their slots, then the correlations
    vs = {m: coeff[m] for m in range(N + 1)}
    vs.update({1 + N + i: z[i] for i in range(n)})
    vs[P["slot_u"]] = u
    run_jobs(vs, P["vjp_jobs"][: P["vjp_fwd_jobs"]])
    for i in range(n):
        vs[P["slot_g0"] + i] = output(P, vs, 1 + i, S)
    run_jobs(vs, P["vjp_jobs"][P["vjp_fwd_jobs"]:])
    gin, gco = vjp_pow_fr(supp, exps, n, coeff, z, u)
    r0 = P["slot_r0"]
    for m in range(N):
        assert vs[r0 + m] == gco[m + 1]
    for i in range(n):
        assert vs[r0 + N + i] == gin[i]


def conj(s):
    return (list(s[0]), [-x for x in s[1]])


def ccorr_fr(u, s):
    """Correlation of complex u with complex s (pairs of Fraction lists)."""
    ur, ui = u
    sr, si = s
    re = [a - b for a, b in zip(corr_fr(ur, sr), corr_fr(ui, si))]
    im = [a + b for a, b in zip(corr_fr(ur, si), corr_fr(ui, sr))]
    return re, im


@pytest.mark.parametrize("powers", [False, True])
@pytest.mark.parametrize("seed", range(3))
def test_complex_program_exact(seed, powers):
    """Complex form of the program: slot s of the real program in 2s (real
    part) and 2s + 1 (imaginary part); outputs 2o and 2o + 1.  The VJP gives
    the correlations of u with the conjugate gradient and monomial series."""
    rng, n, supp, ex = case(3100 + seed, powers)
    N, S = len(supp), 4
    P = pes.jobc_program(supp, n, exponents=ex, complex_series=True, with_vjp=True)
    coeff = [(rand_series(rng, S), rand_series(rng, S)) for _ in range(N + 1)]
    z = [(rand_series(rng, S), rand_series(rng, S)) for _ in range(n)]
    u = (rand_series(rng, S), rand_series(rng, S))
    exps = ex or [[1] * len(s) for s in supp]
    assert P["input_slots"] == 2 * (1 + N + n)

    def inputs():
        slots = {}
        for m in range(N + 1):
            slots[2 * m], slots[2 * m + 1] = coeff[m]
        for i in range(n):
            slots[2 * (1 + N + i)], slots[2 * (1 + N + i) + 1] = z[i]
        return slots

    slots = inputs()
    run_jobs(slots, P["jobs"])
    value, grad, _ = eval_grad_complex_fr(supp, exps, n, coeff, z)
    assert (output(P, slots, 0, S), output(P, slots, 1, S)) == (value[0], value[1])
    for i in range(n):
        assert (output(P, slots, 2 * (1 + i), S), output(P, slots, 2 * (1 + i) + 1, S)) == (grad[i][0], grad[i][1])
    # VJP tables (VJP slot numbers are those of the real program)
    vs = inputs()
    vs[2 * P["slot_u"]], vs[2 * P["slot_u"] + 1] = u
    run_jobs(vs, P["vjp_jobs"][: P["vjp_fwd_jobs"]])
    for i in range(n):
        for part in (0, 1):
            vs[2 * (P["slot_g0"] + i) + part] = output(P, vs, 2 * (1 + i) + part, S)
    run_jobs(vs, P["vjp_jobs"][P["vjp_fwd_jobs"]:])
    one = ([Fraction(1)] + [Fraction(0)] * (S - 1), [Fraction(0)] * S)
    r0 = P["slot_r0"]
    for m, (s_, e_) in enumerate(zip(supp, exps)):
        mono = one
        for v, e in zip(s_, e_):
            for _ in range(e):
                mono = cconv_fr(mono, z[v])
        assert (vs[2 * (r0 + m)], vs[2 * (r0 + m) + 1]) == ccorr_fr(u, conj(mono))
    for i in range(n):
        assert (vs[2 * (r0 + N + i)], vs[2 * (r0 + N + i) + 1]) == ccorr_fr(u, conj(grad[i]))


@pytest.mark.parametrize("powers", [False, True])
@pytest.mark.parametrize("seed", range(3))
def test_system_program_exact(seed, powers):
    """A system of P polynomials: one job table, the constant of polynomial p in
    slot const0 + p, value outputs p < P and Jacobian outputs P + p n + i; the
    VJP with one upstream series per polynomial: coefficient gradients from the
    correlations of u_p with the monomial products, the input gradient the sum
    over p of the correlations of u_p with the Jacobian series."""
    rng = np.random.default_rng(3200 + seed)
    n, S, P = 3, 4, 3
    polys = [synth.random_supports(rng, n, int(rng.integers(0, 4)), 1, n) for _ in range(P)]
    exps = [[[int(e) for e in rng.integers(1, 3, size=len(s_))] for s_ in p_] for p_ in polys] if powers else \
        [[[1] * len(s_) for s_ in p_] for p_ in polys]
    supp = [m for p_ in polys for m in p_]
    flat_ex = [e for pe in exps for e in pe]
    N = len(supp)
    Pr = pes.jobc_program(supp, n, exponents=flat_ex if powers else None, with_vjp=True,
                          polys=[len(p_) for p_ in polys])
    consts = [rand_series(rng, S) for _ in range(P)]
    mcoeff = [rand_series(rng, S) for _ in range(N)]
    z = [rand_series(rng, S) for _ in range(n)]
    u = [rand_series(rng, S) for _ in range(P)]

    def inputs():
        slots = {1 + m: mcoeff[m] for m in range(N)}
        slots.update({1 + N + i: z[i] for i in range(n)})
        slots.update({Pr["const0"] + p: consts[p] for p in range(P)})
        return slots

    slots = inputs()
    run_jobs(slots, Pr["jobs"])
    m0 = 0
    refs = []
    for p, p_ in enumerate(polys):
        coeff = [consts[p]] + mcoeff[m0:m0 + len(p_)]
        value, grad = eval_grad_pow_fr(p_, exps[p], n, coeff, z)
        refs.append((coeff, grad))
        assert output(Pr, slots, p, S) == value
        for i in range(n):
            assert output(Pr, slots, P + p * n + i, S) == grad[i]
        m0 += len(p_)
    # VJP
    vs = inputs()
    for p in range(P):
        vs[Pr["slot_up0"] + p] = u[p]
    run_jobs(vs, Pr["vjp_jobs"][: Pr["vjp_fwd_jobs"]])
    for p in range(P):
        for i in range(n):
            o = P + p * n + i
            if Pr["add_ptr"][o + 1] > Pr["add_ptr"][o]:
                vs[Pr["slot_J0"] + p * n + i] = output(Pr, vs, o, S)
    run_jobs(vs, Pr["vjp_jobs"][Pr["vjp_fwd_jobs"]:])
    m0 = 0
    for p, p_ in enumerate(polys):
        coeff, _ = refs[p]
        ri, rc = vjp_pow_fr(p_, exps[p], n, coeff, z, u[p])
        for m in range(len(p_)):
            assert vs[Pr["slot_r0"] + m0 + m] == rc[m + 1]
        for i in range(n):  # the summands of the input gradient (the sum over p is an addition table)
            o = P + p * n + i
            if Pr["add_ptr"][o + 1] > Pr["add_ptr"][o]:
                assert vs[Pr["slot_rJ0"] + p * n + i] == ri[i]
            else:
                assert all(x == 0 for x in ri[i])
        m0 += len(p_)
