"""Systems of polynomials and their Jacobian matrix (the value and Jacobian
series a Newton step on power series needs) on the GPU, through the C-ABI
(pes_plan_system / pes_eval_system), against the oracle polynomial by
polynomial; bit-identity with one plan per polynomial; the two output layouts;
the VJP with one upstream series per polynomial (pes_vjp, autograd)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_10881_gb300 import pes, synth
from paper_2101_10881_gb300.synth import KS, random_md
from tests.exact import TOL, closed_form_value, normwise_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    pes.build()
    assert _t.cuda.is_available()
    return _t


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def case(k, d, seed, n=7, P=4, N=6, powers=False):
    rng = np.random.default_rng(seed)
    polys, coeffs, exps = [], [], []
    for p in range(P):
        supp = synth.random_supports(rng, n, N + p, 1, 5)
        polys.append(supp)
        coeffs.append(random_md(rng, k, (len(supp) + 1, d + 1)))
        exps.append([[int(e) for e in rng.integers(1, 4, size=len(s))] for s in supp])
    inputs = random_md(rng, k, (n, d + 1))
    return polys, (exps if powers else None), n, coeffs, inputs


def check_against_oracle(torch, polys, exps, n, coeffs, inputs, k, d, **opts):
    sysp = pes.System(polys, n, d, k, exponents=exps, **opts)
    C = dev(torch, np.concatenate(coeffs, axis=1))
    v, J = sysp.eval_system(C, dev(torch, inputs))
    sysp.check()
    v, J = v.cpu().numpy(), J.cpu().numpy()
    for p, supp in enumerate(polys):
        rv, rg = O.eval_grad(supp, n, coeffs[p], inputs, exponents=exps[p] if exps else None)
        assert normwise_err(v[:, p], rv) <= TOL[k], p
        assert normwise_err(J[:, p], rg) <= TOL[k], p
    return sysp, C


@pytest.mark.parametrize("arith", ["int", "fp64"])
@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("d", [0, 9, 40])
def test_system_matches_oracle(torch, k, d, arith):
    polys, _, n, coeffs, inputs = case(k, d, 1100 + 10 * k + d)
    check_against_oracle(torch, polys, None, n, coeffs, inputs, k, d, arith=arith)


@pytest.mark.parametrize("k", [2, 10])
def test_system_with_powers_matches_oracle(torch, k):
    d = 24
    polys, exps, n, coeffs, inputs = case(k, d, 1200 + k, powers=True)
    check_against_oracle(torch, polys, exps, n, coeffs, inputs, k, d)


@pytest.mark.parametrize("powers", [False, True])
@pytest.mark.parametrize("arith", ["int", "fp64"])
def test_system_bit_identical_to_separate_plans(torch, arith, powers):
    """Every monomial's products are the ones its own plan computes, and every
    output is one exact sum rounded once: the system's values and Jacobian rows
    equal, bit for bit, those of one plan per polynomial."""
    k, d = 4, 33
    polys, exps, n, coeffs, inputs = case(k, d, 1300, P=5, powers=powers)
    sysp = pes.System(polys, n, d, k, exponents=exps, arith=arith)
    Z = dev(torch, inputs)
    v, J = sysp.eval_system(dev(torch, np.concatenate(coeffs, axis=1)), Z)
    for p, supp in enumerate(polys):
        plan = pes.Plan(supp, n, d, k, exponents=exps[p] if exps else None, arith=arith)
        pv, pg = plan.eval_grad(dev(torch, coeffs[p]), Z)
        assert torch.equal(v[:, p], pv) and torch.equal(J[:, p], pg), p
    sysp.check()


@pytest.mark.parametrize("k", [1, 5, 8])
def test_system_layouts_agree(torch, k):
    """The matrix layout [k][d+1][P][n] holds exactly the series layout's
    numbers, one P x n matrix per power of t."""
    d = 20
    polys, _, n, coeffs, inputs = case(k, d, 1400 + k)
    sysp = pes.System(polys, n, d, k)
    C, Z = dev(torch, np.concatenate(coeffs, axis=1)), dev(torch, inputs)
    v0, J0 = sysp.eval_system(C, Z, "series")
    v1, J1 = sysp.eval_system(C, Z, "matrix")
    sysp.check()
    assert v1.shape == (k, d + 1, len(polys)) and J1.shape == (k, d + 1, len(polys), n)
    assert torch.equal(v1, v0.permute(0, 2, 1)) and torch.equal(J1, J0.permute(0, 3, 1, 2))
    v2, J2 = sysp.eval_grad(C, Z)
    assert torch.equal(v2, v0) and torch.equal(J2, J0)


def test_system_degenerate_cases(torch):
    """A polynomial with no monomial (its value is its constant, its Jacobian
    row zero), a variable in no polynomial (a zero column), one polynomial
    (the plain plan), d = 0."""
    k, n = 3, 5
    for d in (0, 11):
        rng = np.random.default_rng(1500 + d)
        polys = [[[0, 1], [1, 2, 3]], [], [[0, 3], [3]]]   # x_4 appears nowhere
        coeffs = [random_md(rng, k, (len(s) + 1, d + 1)) for s in polys]
        inputs = random_md(rng, k, (n, d + 1))
        sysp, C = check_against_oracle(torch, polys, None, n, coeffs, inputs, k, d)
        v, J = sysp.eval_system(C, dev(torch, inputs))
        assert torch.equal(v[:, 1], dev(torch, coeffs[1][:, 0]))
        assert not J[:, 1].any() and not J[:, :, 4].any()
        one = pes.System(polys[:1], n, d, k)
        plan = pes.Plan(polys[0], n, d, k)
        Z = dev(torch, inputs)
        v1, J1 = one.eval_system(dev(torch, coeffs[0]), Z)
        pv, pg = plan.eval_grad(dev(torch, coeffs[0]), Z)
        assert torch.equal(v1[:, 0], pv) and torch.equal(J1[:, 0], pg)


def test_system_exp_inputs_closed_form(torch):
    """Inputs z_i = exp(a_i t) and degree-0 coefficients: every value and every
    Jacobian entry is a sum of exponentials with a closed form; one shared
    system of 8 polynomials at k = 10, d = 60 against the oracle, which is
    itself pinned to those closed forms."""
    k, d = 10, 60
    sysc = synth.config4(d, k, seed=3, npoly=8, n=16, N=24, lo=2, hi=6)
    polys = [s for s, _ in sysc.polys]
    coeffs = [c for _, c in sysc.polys]
    check_against_oracle(torch, polys, None, sysc.n, coeffs, sysc.inputs, k, d)


def truncated_value_err(got, ref):
    """Normwise error of limb-major series against exact Fractions."""
    from fractions import Fraction
    g = [sum((Fraction(float(x)) for x in got[:, j]), Fraction(0)) for j in range(got.shape[1])]
    den = max(abs(r) for r in ref)
    return float(max(abs(a - b) for a, b in zip(g, ref)) / den)


def test_system_full_size_sampled(torch):
    """The 64 x 64 system of 512 monomials of 4-16 variables per polynomial at
    d = 152, k = 10, in the matrix layout: for sampled polynomials the first
    four coefficients of the value and of sampled Jacobian entries against the
    oracle on the truncated inputs (coefficient j of a product depends only on
    coefficients 0..j of its factors), and the whole value series against its
    exact closed form (inputs exp(a_i t), degree-0 coefficients)."""
    from fractions import Fraction
    k, d, dd = 10, 152, 3
    sysc = synth.config4(d, k, seed=0)
    polys = [s for s, _ in sysc.polys]
    sysp = pes.System(polys, sysc.n, d, k)
    C = dev(torch, np.concatenate([c for _, c in sysc.polys], axis=1))
    v, J = sysp.eval_system(C, dev(torch, sysc.inputs), "matrix")
    sysp.check()
    v, J = v.cpu().numpy(), J.cpu().numpy()
    z = np.ascontiguousarray(sysc.inputs[:, :, : dd + 1])
    for p in (0, 37, 63):
        supp, c = sysc.polys[p]
        rv, rg = O.eval_grad(supp, sysc.n, np.ascontiguousarray(c[:, :, : dd + 1]), z)
        assert normwise_err(v[:, : dd + 1, p], rv) <= TOL[k]
        for i in (0, 21, 63):
            assert normwise_err(J[:, : dd + 1, p, i], rg[:, i]) <= TOL[k]
        cs = [sum((Fraction(float(x)) for x in c[:, m, 0]), Fraction(0)) for m in range(c.shape[1])]
        ref = closed_form_value(supp, cs, sysc.avals, d)
        assert truncated_value_err(v[:, :, p], ref) <= TOL[k]


def system_vjp(torch, polys, exps, n, coeffs, inputs, u, k, d, **opts):
    sysp = pes.System(polys, n, d, k, exponents=exps, **opts)
    C, Z, U = dev(torch, np.concatenate(coeffs, axis=1)), dev(torch, inputs), dev(torch, u)
    sysp.eval_grad(C, Z)
    gi, gc = sysp.vjp(C, Z, U, reuse_forward=True)
    gi2, gc2 = sysp.vjp(C, Z, U, reuse_forward=False)
    sysp.check()
    assert torch.equal(gi, gi2) and torch.equal(gc, gc2)
    return sysp, gi.cpu().numpy(), gc.cpu().numpy()


@pytest.mark.parametrize("k", [1, 2, 4])
def test_system_vjp_exact_tiny(torch, k):
    """L = sum_p <u_p, v_p> on a tiny system: grad_input (summed over the
    polynomials) and grad_coeff against exact rational arithmetic."""
    from tests.exact import normwise_err_fr, series_fractions, vjp_fr
    d, n = 5, 4
    rng = np.random.default_rng(1600 + k)
    polys = [[[0, 1], [1, 2, 3]], [[2], [0, 3]], [[0, 1, 2, 3]]]
    coeffs = [random_md(rng, k, (len(p_) + 1, d + 1)) for p_ in polys]
    inputs = random_md(rng, k, (n, d + 1))
    u = random_md(rng, k, (len(polys), d + 1))
    _, gi, gc = system_vjp(torch, polys, None, n, coeffs, inputs, u, k, d)
    zf = series_fractions(inputs)
    gin_ref = np.zeros((n, d + 1), dtype=object)
    row = 0
    for p, p_ in enumerate(polys):
        gin, gco = vjp_fr(p_, n, series_fractions(coeffs[p]), zf, series_fractions(u[:, p]))
        gin_ref = gin_ref + np.array(gin, dtype=object)
        assert normwise_err_fr(gc[:, row:row + len(p_) + 1], gco) <= TOL[k]
        row += len(p_) + 1
    assert normwise_err_fr(gi, gin_ref) <= TOL[k]


@pytest.mark.parametrize("powers", [False, True])
@pytest.mark.parametrize("k", [2, 10])
def test_system_vjp_matches_oracle(torch, k, powers):
    """Against the oracle's VJP polynomial by polynomial: grad_coeff rows
    exactly as each polynomial's own; grad_input the sum over the polynomials
    (the oracle's per-polynomial results are each rounded, so their exact sum
    is within P times the tolerance)."""
    from tests.exact import normwise_err_fr, series_fractions
    d = 30
    polys, exps, n, coeffs, inputs = case(k, d, 1700 + k, powers=powers)
    u = random_md(np.random.default_rng(1701 + k), k, (len(polys), d + 1))
    _, gi, gc = system_vjp(torch, polys, exps, n, coeffs, inputs, u, k, d)
    gin_ref = np.zeros((n, d + 1), dtype=object)
    row = 0
    for p, p_ in enumerate(polys):
        ri, rc = O.vjp(p_, n, coeffs[p], inputs, np.ascontiguousarray(u[:, p]), exponents=exps[p] if exps else None)
        gin_ref = gin_ref + series_fractions(ri)
        assert normwise_err(gc[:, row:row + len(p_) + 1], rc) <= TOL[k]
        row += len(p_) + 1
    assert normwise_err_fr(gi, gin_ref) <= len(polys) * TOL[k]


def test_system_autograd_matches_separate_plans(torch):
    """torch.autograd through a system plan (poly_eval with one upstream
    series per polynomial) against the same loss through one plan per
    polynomial: L = sum_p sum_j v_pj^2."""
    from paper_2101_10881_gb300.autograd import poly_eval
    from tests.exact import normwise_err_fr, series_fractions
    k, d = 3, 25
    polys, _, n, coeffs, inputs = case(k, d, 1800)
    sysp = pes.System(polys, n, d, k)
    C = dev(torch, np.concatenate(coeffs, axis=1)).requires_grad_(True)
    Z = dev(torch, inputs).requires_grad_(True)
    v = poly_eval(C, Z, sysp)
    assert v.shape == (k, len(polys), d + 1)
    v.backward(2 * v.detach())
    sysp.check()
    gz_ref = np.zeros((n, d + 1), dtype=object)
    row = 0
    for p, p_ in enumerate(polys):
        plan = pes.Plan(p_, n, d, k)
        Cp = dev(torch, coeffs[p]).requires_grad_(True)
        Zp = dev(torch, inputs).requires_grad_(True)
        vp = poly_eval(Cp, Zp, plan)
        assert torch.equal(vp.detach(), v.detach()[:, p])
        vp.backward(2 * vp.detach())
        assert torch.equal(Cp.grad, C.grad[:, row:row + len(p_) + 1])
        gz_ref = gz_ref + series_fractions(Zp.grad.cpu().numpy())
        row += len(p_) + 1
    assert normwise_err_fr(Z.grad.cpu().numpy(), gz_ref) <= len(polys) * TOL[k]


def test_system_of_constants(torch):
    """Every polynomial a constant (no monomial at all): values are the
    constants, the Jacobian is zero, the VJP gives u_p for every constant and
    a zero input gradient."""
    k, d, n = 2, 9, 3
    rng = np.random.default_rng(1900)
    coeffs = [random_md(rng, k, (1, d + 1)) for _ in range(3)]
    inputs = random_md(rng, k, (n, d + 1))
    u = random_md(rng, k, (3, d + 1))
    sysp, gi, gc = system_vjp(torch, [[], [], []], None, n, coeffs, inputs, u, k, d)
    v, J = sysp.eval_system(dev(torch, np.concatenate(coeffs, axis=1)), dev(torch, inputs))
    sysp.check()
    assert np.array_equal(v.cpu().numpy(), np.concatenate(coeffs, axis=1))
    assert not J.any() and not gi.any()
    assert np.array_equal(gc, u)


def test_system_tiled_bit_identical(torch):
    """A system through the tiled kernel (forced tiles of 24 coefficients):
    values, Jacobian in both layouts and the VJP give the whole-series bits."""
    k, d = 4, 75
    polys, exps, n, coeffs, inputs = case(k, d, 2000, powers=True)
    u = random_md(np.random.default_rng(2001), k, (len(polys), d + 1))
    C, Z, U = dev(torch, np.concatenate(coeffs, axis=1)), dev(torch, inputs), dev(torch, u)
    out = []
    for tile in (0, 24):
        sysp = pes.System(polys, n, d, k, exponents=exps, tile=tile)
        assert sysp.info()["tile"] == tile
        v0, J0 = sysp.eval_system(C, Z, "series")
        v1, J1 = sysp.eval_system(C, Z, "matrix")
        gi, gc = sysp.vjp(C, Z, U, reuse_forward=True)
        sysp.check()
        out.append((v0, J0, v1, J1, gi, gc))
    for a, b in zip(*out):
        assert torch.equal(a, b)
