"""The autograd Function: gradients with respect to coefficient and input
series (k-double convention) against the oracle's VJP, and the three ways the
backward obtains the forward products (live workspace, snapshot kept under a
memory budget, recomputation) give identical results."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_10881_gb300 import pes, synth
from paper_2101_10881_gb300.synth import random_md
from tests.exact import TOL, normwise_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    pes.build()
    assert _t.cuda.is_available()
    return _t


def case(k, seed, n=7, N=11, d=20):
    rng = np.random.default_rng(seed)
    supp = synth.random_supports(rng, n, N, 1, 5)
    return supp, n, d, random_md(rng, k, (N + 1, d + 1)), random_md(rng, k, (n, d + 1))


@pytest.mark.parametrize("k", [2, 4, 8])
def test_autograd_matches_oracle_vjp(torch, k):
    from paper_2101_10881_gb300.autograd import poly_eval
    supp, n, d, coeff, inputs = case(k, 500 + k)
    plan = pes.Plan(supp, n, d, k)
    C = torch.from_numpy(coeff).cuda().requires_grad_(True)
    Z = torch.from_numpy(inputs).cuda().requires_grad_(True)
    v = poly_eval(C, Z, plan)
    v.backward(2 * v.detach())  # L = sum_j v_j^2 in k-double: u = 2 v
    u = 2 * v.detach().cpu().numpy()
    ri, rc = O.vjp(supp, n, coeff, inputs, u)
    assert normwise_err(Z.grad.cpu().numpy(), ri) <= TOL[k]
    assert normwise_err(C.grad.cpu().numpy(), rc) <= TOL[k]
    rv = O.eval_grad(supp, n, coeff, inputs, grad=False)
    assert normwise_err(v.detach().cpu().numpy(), rv) <= TOL[k]


def test_backward_paths_agree(torch):
    """Live workspace, snapshot under a budget, and recomputation."""
    from paper_2101_10881_gb300.autograd import poly_eval
    k = 4
    supp, n, d, coeff, inputs = case(k, 77)
    _, _, _, coeff2, inputs2 = case(k, 78)
    plan = pes.Plan(supp, n, d, k)
    grads = []
    for mode in ("live", "snapshot", "recompute"):
        C = torch.from_numpy(coeff).cuda().requires_grad_(True)
        Z = torch.from_numpy(inputs).cuda().requires_grad_(True)
        budget = 1 << 40 if mode == "snapshot" else None
        v = poly_eval(C, Z, plan, memory_budget=budget)
        if mode != "live":
            # another evaluation on the same plan overwrites its workspace
            poly_eval(torch.from_numpy(coeff2).cuda(), torch.from_numpy(inputs2).cuda(), plan)
        u = torch.from_numpy(random_md(np.random.default_rng(5), k, (d + 1,))).cuda()
        v.backward(u)
        grads.append((C.grad.cpu().numpy(), Z.grad.cpu().numpy()))
    for gc, gi in grads[1:]:
        assert np.array_equal(gc, grads[0][0]) and np.array_equal(gi, grads[0][1])
