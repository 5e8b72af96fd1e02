"""Complex coefficient and input series on the GPU (pes_plan_complex) against
the oracle: every complex product four real ones combined exactly by add and
subtract jobs, real and imaginary parts summed separately; the VJP (gradients
with respect to real and imaginary parts, correlations with conjugate series)
and autograd."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_10881_gb300 import pes, synth
from paper_2101_10881_gb300.synth import KS, random_md
from tests.exact import TOL, normwise_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    pes.build()
    assert _t.cuda.is_available()
    return _t


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def case(k, d, seed, n=5, N=7, powers=False):
    rng = np.random.default_rng(seed)
    supp = synth.random_supports(rng, n, N, 1, 4)
    ex = [[int(e) for e in rng.integers(1, 4, size=len(s))] for s in supp] if powers else None
    coeff = np.stack([random_md(rng, k, (N + 1, d + 1)), random_md(rng, k, (N + 1, d + 1))])
    inputs = np.stack([random_md(rng, k, (n, d + 1)), random_md(rng, k, (n, d + 1))])
    return supp, ex, n, coeff, inputs


@pytest.mark.parametrize("arith", ["int", "fp64"])
@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("d", [0, 9, 40])
def test_complex_matches_oracle(torch, k, d, arith):
    supp, ex, n, coeff, inputs = case(k, d, 1200 + 10 * k + d, powers=(d == 9))
    plan = pes.Plan(supp, n, d, k, exponents=ex, complex_series=True, arith=arith)
    assert plan.info()["complex_series"] == 1
    v, g = plan.eval_grad(dev(torch, coeff), dev(torch, inputs))
    plan.check()
    rv, rg = O.eval_grad_complex(supp, n, coeff, inputs, exponents=ex)
    v, g = v.cpu().numpy(), g.cpu().numpy()
    for part in (0, 1):
        assert normwise_err(v[part], rv[part]) <= TOL[k]
        assert normwise_err(g[part], rg[part]) <= TOL[k]


def test_complex_high_degree(torch):
    k, d = 10, 152
    supp, ex, n, coeff, inputs = case(k, d, 1250, n=3, N=3)
    plan = pes.Plan(supp, n, d, k, complex_series=True)
    v, g = plan.eval_grad(dev(torch, coeff), dev(torch, inputs))
    plan.check()
    rv, rg = O.eval_grad_complex(supp, n, coeff, inputs)
    v, g = v.cpu().numpy(), g.cpu().numpy()
    for part in (0, 1):
        assert normwise_err(v[part], rv[part]) <= TOL[k]
        assert normwise_err(g[part], rg[part]) <= TOL[k]


def test_complex_with_zero_imaginary_parts_is_the_real_plan(torch):
    k, d = 4, 30
    rng = np.random.default_rng(1260)
    n = 6
    supp = synth.random_supports(rng, n, 8, 1, 5)
    coeff = random_md(rng, k, (len(supp) + 1, d + 1))
    inputs = random_md(rng, k, (n, d + 1))
    v, g = pes.Plan(supp, n, d, k).eval_grad(dev(torch, coeff), dev(torch, inputs))
    cv, cg = pes.Plan(supp, n, d, k, complex_series=True).eval_grad(
        dev(torch, np.stack([coeff, 0 * coeff])), dev(torch, np.stack([inputs, 0 * inputs])))
    assert torch.equal(cv[0], v) and torch.equal(cg[0], g)
    assert not cv[1].any() and not cg[1].any()


def test_complex_conjugation(torch):
    k, d = 3, 20
    supp, _, n, coeff, inputs = case(k, d, 1270)
    plan = pes.Plan(supp, n, d, k, complex_series=True)
    v, g = plan.eval_grad(dev(torch, coeff), dev(torch, inputs))
    cc, ci = coeff.copy(), inputs.copy()
    cc[1], ci[1] = -cc[1], -ci[1]
    w, h = plan.eval_grad(dev(torch, cc), dev(torch, ci))
    assert torch.equal(w[0], v[0]) and torch.equal(w[1], -v[1])
    assert torch.equal(h[0], g[0]) and torch.equal(h[1], -g[1])


def complex_vjp(torch, plan, coeff, inputs, u):
    C, Z, U = dev(torch, coeff), dev(torch, inputs), dev(torch, u)
    plan.eval_grad(C, Z)
    gi, gc = plan.vjp(C, Z, U, reuse_forward=True)
    gi2, gc2 = plan.vjp(C, Z, U, reuse_forward=False)
    plan.check()
    assert torch.equal(gi, gi2) and torch.equal(gc, gc2)
    return gi.cpu().numpy(), gc.cpu().numpy()


@pytest.mark.parametrize("powers", [False, True])
@pytest.mark.parametrize("arith", ["int", "fp64"])
@pytest.mark.parametrize("k", [1, 2, 5, 10])
def test_complex_vjp_matches_oracle(torch, k, arith, powers):
    """The derivatives of L = sum_j Re u_j Re v_j + Im u_j Im v_j with respect to
    the real and imaginary parts of every input and coefficient series
    (correlations with the conjugate series), with and without reuse of the
    forward products, against the oracle."""
    d = 24
    supp, ex, n, coeff, inputs = case(k, d, 1300 + k, powers=powers)
    u = np.stack([random_md(np.random.default_rng(1301 + k), k, (d + 1,)),
                  random_md(np.random.default_rng(1302 + k), k, (d + 1,))])
    plan = pes.Plan(supp, n, d, k, exponents=ex, complex_series=True, arith=arith)
    gi, gc = complex_vjp(torch, plan, coeff, inputs, u)
    ri, rc = O.vjp_complex(supp, n, coeff, inputs, u, exponents=ex)
    for part in (0, 1):
        assert normwise_err(gi[part], ri[part]) <= TOL[k]
        assert normwise_err(gc[part], rc[part]) <= TOL[k]


def test_complex_vjp_with_zero_imaginary_parts_is_the_real_vjp(torch):
    """Zero imaginary parts everywhere: the real parts of the gradients are the
    real plan's VJP bit for bit, the imaginary parts zero."""
    k, d = 4, 30
    supp, _, n, coeff, inputs = case(k, d, 1310)
    u = random_md(np.random.default_rng(1311), k, (d + 1,))
    real = pes.Plan(supp, n, d, k)
    ri, rc = complex_vjp(torch, real, coeff[0], inputs[0], u)
    cplx = pes.Plan(supp, n, d, k, complex_series=True)
    gi, gc = complex_vjp(torch, cplx, np.stack([coeff[0], 0 * coeff[0]]), np.stack([inputs[0], 0 * inputs[0]]),
                         np.stack([u, 0 * u]))
    assert np.array_equal(gi[0], ri) and np.array_equal(gc[0], rc)
    assert not gi[1].any() and not gc[1].any()


def test_complex_autograd(torch):
    """torch.autograd through a complex plan (pairs of real tensors): the
    backward of L = sum of the squares of every real and imaginary part of the
    value series against the oracle's VJP with u = 2 v."""
    from paper_2101_10881_gb300.autograd import poly_eval
    k, d = 3, 20
    supp, _, n, coeff, inputs = case(k, d, 1320)
    plan = pes.Plan(supp, n, d, k, complex_series=True)
    C = dev(torch, coeff).requires_grad_(True)
    Z = dev(torch, inputs).requires_grad_(True)
    v = poly_eval(C, Z, plan)
    assert v.shape == (2, k, d + 1)
    v.backward(2 * v.detach())
    plan.check()
    ri, rc = O.vjp_complex(supp, n, coeff, inputs, 2 * v.detach().cpu().numpy())
    for part in (0, 1):
        assert normwise_err(Z.grad.cpu().numpy()[part], ri[part]) <= TOL[k]
        assert normwise_err(C.grad.cpu().numpy()[part], rc[part]) <= TOL[k]


def test_complex_vjp_tiled_bit_identical(torch):
    """The tiled kernel (correlation and add / subtract jobs per output tile)
    gives the whole-series kernel's bits for the complex VJP."""
    k, d = 2, 61
    supp, ex, n, coeff, inputs = case(k, d, 1330, powers=True)
    u = np.stack([random_md(np.random.default_rng(1331), k, (d + 1,)),
                  random_md(np.random.default_rng(1332), k, (d + 1,))])
    out = [complex_vjp(torch, pes.Plan(supp, n, d, k, exponents=ex, complex_series=True, tile=t), coeff, inputs, u)
           for t in (0, 16)]
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
