"""Complex coefficient and input series on the GPU (pes_plan_complex) against
the oracle: every complex product four real ones combined exactly by add and
subtract jobs, real and imaginary parts summed separately."""
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


def test_complex_plan_has_no_vjp(torch):
    k, d = 2, 5
    supp, _, n, coeff, inputs = case(k, d, 1280)
    plan = pes.Plan(supp, n, d, k, complex_series=True)
    with pytest.raises(pes.PesError) as e:
        plan.vjp(dev(torch, coeff), dev(torch, inputs), dev(torch, np.zeros((2, k, d + 1))))
    assert e.value.code == 1
