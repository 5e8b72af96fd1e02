"""One polynomial split over ranks, on the GPU: the ranks' plans run one after
another on this one GPU (no kernel of one rank waits on another), the exchange
is done with the same integer operations the collectives perform (elementwise
maximum of the grids, sum of the digit sums), and every rank's rounded result
must equal one plan of the whole polynomial bit for bit, and the oracle within
the per-k tolerance."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_10881_gb300 import pes, synth
from paper_2101_10881_gb300.shard import ShardPlan, combine_host
from paper_2101_10881_gb300.synth import random_md
from tests.exact import TOL, normwise_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    pes.build()
    assert _t.cuda.is_available()
    return _t


def cases():
    rng = np.random.default_rng(321)
    p2 = synth.supports_p2(n=24, N=12, m=8, seed=5)
    p3 = synth.supports_p3(20)
    mixed = synth.random_supports(rng, 9, 23, 1, 6)
    pw = [[int(e) for e in rng.integers(1, 4, size=len(s))] for s in mixed]
    return [("p2-like k=10", p2, 24, 40, 10, None), ("p3 k=4", p3, 20, 30, 4, None),
            ("mixed k=2 powers", mixed, 9, 25, 2, pw), ("mixed k=3", mixed, 9, 152, 3, None)]


@pytest.mark.parametrize("case", range(4))
@pytest.mark.parametrize("world", [2, 3])
def test_shards_equal_one_plan(torch, case, world):
    name, supports, n, d, k, exps = cases()[case]
    rng = np.random.default_rng(1000 + case)
    coeff = random_md(rng, k, (len(supports) + 1, d + 1))
    inputs = random_md(rng, k, (n, d + 1))
    C = torch.from_numpy(coeff).cuda()
    Z = torch.from_numpy(inputs).cuda()
    whole = pes.Plan(supports, n, d, k, exponents=exps, with_vjp=False)
    v0, g0 = whole.eval_grad(C, Z)
    whole.check()

    shards = [ShardPlan(supports, n, d, k, world, r, exponents=exps) for r in range(world)]
    assert shards[0].m_begin == 0 and shards[-1].m_end == len(supports)
    Cr = [s.coeff_of(C) for s in shards]
    grids = [s.plan.partial_grids(c, Z).clone() for s, c in zip(shards, Cr)]
    common = grids[0]
    for g in grids[1:]:
        common = torch.maximum(common, g)
    accs = [s.plan.partial_sums(common).clone() for s in shards]
    total = sum(accs[1:], accs[0].clone())
    for s in shards:
        v, g = s.plan.round_sums(common, total)
        s.plan.check()
        assert torch.equal(v, v0) and torch.equal(g, g0), name
    # the host twin of the rounding gives the same bits
    hv, hg = combine_host(k, n, d, [(common.cpu().numpy(), a.cpu().numpy()) for a in accs])
    assert np.array_equal(hv, v0.cpu().numpy()) and np.array_equal(hg, g0.cpu().numpy())
    if d <= 40:
        rv, rg = O.eval_grad(supports, n, coeff, inputs, exponents=exps)
        assert normwise_err(v0.cpu().numpy(), rv) <= TOL[k] and normwise_err(g0.cpu().numpy(), rg) <= TOL[k]


def test_partial_calls_reject_complex_plans(torch):
    plan = pes.Plan([[0, 1]], 2, 4, 2, complex_series=True)
    C = torch.zeros((2, 2, 2, 5), dtype=torch.float64, device="cuda")
    Z = torch.zeros((2, 2, 2, 5), dtype=torch.float64, device="cuda")
    grids = torch.empty((3, 5), dtype=torch.int32, device="cuda")
    import ctypes
    rc = pes.lib().pes_partial_grids(plan.handle, ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(Z.data_ptr()),
                                     ctypes.c_void_p(grids.data_ptr()), None)
    assert rc == 1


def test_autotuned_shards_equal_one_plan(torch):
    """Rank plans built with autotune tune their launch shape (parts per job
    included) on the first pes_partial_grids call; the exchanged result is
    still one plan's bits."""
    supports = synth.supports_p2(n=32, N=8, m=16, seed=9)
    n, d, k, world = 32, 152, 10, 2
    rng = np.random.default_rng(77)
    C = torch.from_numpy(random_md(rng, k, (len(supports) + 1, d + 1))).cuda()
    Z = torch.from_numpy(random_md(rng, k, (n, d + 1))).cuda()
    whole = pes.Plan(supports, n, d, k, with_vjp=False)
    v0, g0 = whole.eval_grad(C, Z)
    shards = [ShardPlan(supports, n, d, k, world, r, autotune=True) for r in range(world)]
    grids = [s.plan.partial_grids(s.coeff_of(C), Z).clone() for s in shards]
    common = torch.maximum(grids[0], grids[1])
    total = sum((s.plan.partial_sums(common).clone() for s in shards[1:]), shards[0].plan.partial_sums(common).clone())
    for s in shards:
        v, g = s.plan.round_sums(common, total)
        s.plan.check()
        assert torch.equal(v, v0) and torch.equal(g, g0)
        assert s.plan.info()["split"] in (1, 2, 4, 8, 16)
