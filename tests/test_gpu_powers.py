"""Monomials with positive powers (Sec. 3) on the GPU, through the C-ABI
(pes_plan_powers), against the oracle: value, gradient and VJP, both
multiply-accumulate pipes, and the autograd Function on a plan with powers."""
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


def case(k, d, seed, n=6, N=9, hi=4):
    rng = np.random.default_rng(seed)
    supp = synth.random_supports(rng, n, N, 1, 5)
    ex = [[int(e) for e in rng.integers(1, hi + 1, size=len(s))] for s in supp]
    return supp, ex, n, random_md(rng, k, (N + 1, d + 1)), random_md(rng, k, (n, d + 1))


@pytest.mark.parametrize("arith", ["int", "fp64"])
@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("d", [0, 7, 40])
def test_powers_match_oracle(torch, k, d, arith):
    supp, ex, n, coeff, inputs = case(k, d, 900 + 10 * k + d)
    plan = pes.Plan(supp, n, d, k, exponents=ex, arith=arith)
    v, g = plan.eval_grad(dev(torch, coeff), dev(torch, inputs))
    plan.check()
    rv, rg = O.eval_grad(supp, n, coeff, inputs, exponents=ex)
    assert normwise_err(v.cpu().numpy(), rv) <= TOL[k]
    assert normwise_err(g.cpu().numpy(), rg) <= TOL[k]


def test_powers_exp_inputs_high_degree(torch):
    """z_i = exp(a_i t) at d = 100, k = 10: high powers of series whose
    coefficients fall like 1/j!, against the oracle."""
    k, d, n = 10, 100, 5
    rng = np.random.default_rng(950)
    avals = [float(a) for a in rng.uniform(-1, 1, size=n)]
    inputs = synth.exp_inputs(avals, d, k)
    supp = [[0, 1], [1, 2, 4], [0, 3], [2]]
    ex = [[5, 2], [1, 3, 2], [4, 4], [6]]
    coeff = synth.scalar_coeffs(rng, k, len(supp), d)
    plan = pes.Plan(supp, n, d, k, exponents=ex)
    v, g = plan.eval_grad(dev(torch, coeff), dev(torch, inputs))
    plan.check()
    rv, rg = O.eval_grad(supp, n, coeff, inputs, exponents=ex)
    assert normwise_err(v.cpu().numpy(), rv) <= TOL[k]
    assert normwise_err(g.cpu().numpy(), rg) <= TOL[k]


@pytest.mark.parametrize("k", [2, 8])
def test_powers_vjp_matches_oracle(torch, k):
    d = 30
    supp, ex, n, coeff, inputs = case(k, d, 960 + k)
    u = random_md(np.random.default_rng(961 + k), k, (d + 1,))
    plan = pes.Plan(supp, n, d, k, exponents=ex)
    C, Z, U = dev(torch, coeff), dev(torch, inputs), dev(torch, u)
    plan.eval_grad(C, Z)
    gi, gc = plan.vjp(C, Z, U, reuse_forward=True)
    gi2, gc2 = plan.vjp(C, Z, U, reuse_forward=False)
    plan.check()
    ri, rc = O.vjp(supp, n, coeff, inputs, u, exponents=ex)
    assert normwise_err(gi.cpu().numpy(), ri) <= TOL[k]
    assert normwise_err(gc.cpu().numpy(), rc) <= TOL[k]
    assert torch.equal(gi, gi2) and torch.equal(gc, gc2)


def test_powers_autograd(torch):
    from paper_2101_10881_gb300.autograd import poly_eval
    k, d = 4, 20
    supp, ex, n, coeff, inputs = case(k, d, 970)
    plan = pes.Plan(supp, n, d, k, exponents=ex)
    C = dev(torch, coeff).requires_grad_(True)
    Z = dev(torch, inputs).requires_grad_(True)
    v = poly_eval(C, Z, plan)
    v.backward(2 * v.detach())
    u = 2 * v.detach().cpu().numpy()
    ri, rc = O.vjp(supp, n, coeff, inputs, u, exponents=ex)
    assert normwise_err(Z.grad.cpu().numpy(), ri) <= TOL[k]
    assert normwise_err(C.grad.cpu().numpy(), rc) <= TOL[k]


def test_exponents_one_same_bits_as_plain_plan(torch):
    k, d = 3, 25
    supp, _, n, coeff, inputs = case(k, d, 980)
    ones = [[1] * len(s) for s in supp]
    C, Z = dev(torch, coeff), dev(torch, inputs)
    v1, g1 = pes.Plan(supp, n, d, k).eval_grad(C, Z)
    v2, g2 = pes.Plan(supp, n, d, k, exponents=ones).eval_grad(C, Z)
    assert torch.equal(v1, v2) and torch.equal(g1, g2)


def test_invalid_exponents_rejected(torch):
    for bad in ([[0, 1]], [[1, 65]]):
        with pytest.raises(pes.PesError) as e:
            pes.Plan([[0, 1]], 2, 4, 2, exponents=bad)
        assert e.value.code == 1


def test_batch_with_powers_matches_single_plans(torch):
    """Batched instances with powers (pes_plan_batch_powers), mixed degrees:
    every instance equals its own plan bit for bit and the oracle within
    tolerance."""
    k = 3
    rng = np.random.default_rng(970)
    insts, probs, exps = [], [], []
    for b, d in enumerate([0, 7, 31, 152, 60]):
        n = int(rng.integers(3, 7))
        N = int(rng.integers(1, 7))
        supp = synth.random_supports(rng, n, N, 1, min(n, 4))
        ex = [[int(e) for e in rng.integers(1, 4, size=len(s))] for s in supp]
        probs.append(synth.Problem(f"b{b}", n, d, k, supp, random_md(rng, k, (N + 1, d + 1)),
                                   random_md(rng, k, (n, d + 1))))
        insts.append((supp, n, d))
        exps.append(ex)
    B = pes.Batch(insts, k, exponents=exps)
    C = dev(torch, np.concatenate([p.coeff.ravel() for p in probs]))
    Z = dev(torch, np.concatenate([p.inputs.ravel() for p in probs]))
    ln = B.lengths()
    V = torch.empty(ln["value"], dtype=torch.float64, device="cuda")
    G = torch.empty(ln["grad"], dtype=torch.float64, device="cuda")
    for _ in range(2):
        B.eval_grad(C, Z, V, G)
    B.check()
    V, G = V.cpu().numpy(), G.cpu().numpy()
    for b, p in enumerate(probs):
        plan = pes.Plan(p.supports, p.n, p.d, k, exponents=exps[b], with_vjp=False)
        sv, sg = plan.eval_grad(dev(torch, p.coeff), dev(torch, p.inputs))
        v = V[B.value_off[b]:B.value_off[b + 1]].reshape(k, p.d + 1)
        g = G[B.grad_off[b]:B.grad_off[b + 1]].reshape(k, p.n, p.d + 1)
        assert np.array_equal(v, sv.cpu().numpy()) and np.array_equal(g, sg.cpu().numpy())
        rv, rg = O.eval_grad(p.supports, p.n, p.coeff, p.inputs, exponents=exps[b])
        assert normwise_err(v, rv) <= TOL[k] and normwise_err(g, rg) <= TOL[k]
