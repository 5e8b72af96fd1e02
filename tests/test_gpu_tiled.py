"""Degrees beyond the shared-memory staging of whole series: the tiled kernel
(every job split into output tiles, each accumulated tile pair by tile pair
from staged tiles of its operands) through the C-ABI.  At degrees both kernels
take, the tiled kernel gives the whole-series kernel's bits (the same exact
sums cut to the same digits); beyond them, every output against the oracle."""
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


def case(k, d, seed, n=6, N=8, hi=5):
    rng = np.random.default_rng(seed)
    supp = synth.random_supports(rng, n, N, 1, hi)
    return supp, n, random_md(rng, k, (N + 1, d + 1)), random_md(rng, k, (n, d + 1))


@pytest.mark.parametrize("arith", ["int", "fp64"])
@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("d,tile", [(0, 16), (5, 16), (37, 16), (130, 32), (250, 64)])
def test_tiles_bit_identical_to_whole_series(torch, k, d, tile, arith):
    """Ragged last tiles, a degree below one tile, many tiles per job: value
    and gradient equal the whole-series kernel's bit for bit."""
    supp, n, coeff, inputs = case(k, d, 5000 + 10 * k + d)
    C, Z = dev(torch, coeff), dev(torch, inputs)
    whole = pes.Plan(supp, n, d, k, arith=arith)
    tiled = pes.Plan(supp, n, d, k, arith=arith, tile=tile)
    assert whole.info()["tile"] == 0 and tiled.info()["tile"] == tile
    v0, g0 = whole.eval_grad(C, Z)
    v1, g1 = tiled.eval_grad(C, Z)
    tiled.check()
    assert torch.equal(v0, v1) and torch.equal(g0, g1)


@pytest.mark.parametrize("k", [2, 10])
def test_tiled_vjp_bit_identical(torch, k):
    """The correlations of the VJP (transposed convolutions, tiled from the
    other end) and the monomial products, both with and without reuse of the
    forward products."""
    d = 90
    supp, n, coeff, inputs = case(k, d, 5100 + k)
    u = random_md(np.random.default_rng(5101 + k), k, (d + 1,))
    C, Z, U = dev(torch, coeff), dev(torch, inputs), dev(torch, u)
    out = []
    for tile in (0, 24):
        plan = pes.Plan(supp, n, d, k, tile=tile)
        plan.eval_grad(C, Z)
        gi, gc = plan.vjp(C, Z, U, reuse_forward=True)
        gi2, gc2 = plan.vjp(C, Z, U, reuse_forward=False)
        plan.check()
        assert torch.equal(gi, gi2) and torch.equal(gc, gc2)
        out.append((gi, gc))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    ri, rc = O.vjp(supp, n, coeff, inputs, u)
    assert normwise_err(out[1][0].cpu().numpy(), ri) <= TOL[k]
    assert normwise_err(out[1][1].cpu().numpy(), rc) <= TOL[k]


def test_tiled_complex_and_powers_bit_identical(torch):
    """Complex series (the exact add / subtract jobs run per tile) and
    monomials with powers (the power table and common factors)."""
    k, d = 4, 70
    rng = np.random.default_rng(5200)
    supp = synth.random_supports(rng, 5, 6, 1, 4)
    ex = [[int(e) for e in rng.integers(1, 4, size=len(s))] for s in supp]
    coeff = np.stack([random_md(rng, k, (len(supp) + 1, d + 1)) for _ in range(2)])
    inputs = np.stack([random_md(rng, k, (5, d + 1)) for _ in range(2)])
    C, Z = dev(torch, coeff), dev(torch, inputs)
    res = []
    for tile in (0, 16):
        plan = pes.Plan(supp, 5, d, k, exponents=ex, complex_series=True, tile=tile)
        res.append(plan.eval_grad(C, Z))
        plan.check()
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])
    rv, rg = O.eval_grad_complex(supp, 5, coeff, inputs, exponents=ex)
    v, g = res[1][0].cpu().numpy(), res[1][1].cpu().numpy()
    for part in (0, 1):  # real, imaginary: each a k-limb array
        assert normwise_err(v[part], rv[part]) <= TOL[k]
        assert normwise_err(g[part], rg[part]) <= TOL[k]


@pytest.mark.parametrize("k,d", [(10, 700), (8, 1000), (5, 1200), (3, 1500), (2, 3000), (1, 8191)])
def test_large_degree_matches_oracle(torch, k, d):
    """Degrees the whole-series kernel cannot take, chosen by the automatic
    rule, every output coefficient against the oracle."""
    rng = np.random.default_rng(5300 + k)
    supp, n = [[0, 1], [1, 2, 3], [0, 3]], 4
    coeff = random_md(rng, k, (len(supp) + 1, d + 1))
    inputs = random_md(rng, k, (n, d + 1))
    plan = pes.Plan(supp, n, d, k)
    assert plan.info()["tile"] == 128 and plan.info()["arith_name"] == "int"
    v, g = plan.eval_grad(dev(torch, coeff), dev(torch, inputs))
    plan.check()
    rv, rg = O.eval_grad(supp, n, coeff, inputs)
    assert normwise_err(v.cpu().numpy(), rv) <= TOL[k]
    assert normwise_err(g.cpu().numpy(), rg) <= TOL[k]


def test_largest_degree(torch):
    """d = 16383, the API's largest degree, at k = 1 (128 tiles per job) against
    the oracle; fp64 pipe at k = 2 beyond its whole-series limit."""
    rng = np.random.default_rng(5400)
    supp, n = [[0, 1], [1]], 2
    for k, d, arith in ((1, 16383, "int"), (2, 1500, "fp64")):
        coeff = random_md(rng, k, (3, d + 1))
        inputs = random_md(rng, k, (n, d + 1))
        plan = pes.Plan(supp, n, d, k, arith=arith)
        assert plan.info()["tile"] == 128
        v, g = plan.eval_grad(dev(torch, coeff), dev(torch, inputs))
        plan.check()
        rv, rg = O.eval_grad(supp, n, coeff, inputs)
        assert normwise_err(v.cpu().numpy(), rv) <= TOL[k]
        assert normwise_err(g.cpu().numpy(), rg) <= TOL[k]


def test_batch_with_tiled_group(torch):
    """A batch whose large-degree instances run in a tiled group beside the
    whole-series groups: every instance equals its own plan bit for bit."""
    k = 2
    rng = np.random.default_rng(5500)
    insts, probs = [], []
    for b, d in enumerate([7, 63, 1500, 152, 2100]):
        n = int(rng.integers(3, 7))
        N = int(rng.integers(1, 6))
        supp = synth.random_supports(rng, n, N, 1, min(n, 4))
        probs.append(synth.Problem(f"b{b}", n, d, k, supp, random_md(rng, k, (N + 1, d + 1)),
                                   random_md(rng, k, (n, d + 1))))
        insts.append((supp, n, d))
    B = pes.Batch(insts, k)
    assert B.info()["tile"] == 128
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
        plan = pes.Plan(p.supports, p.n, p.d, k, with_vjp=False)
        sv, sg = plan.eval_grad(dev(torch, p.coeff), dev(torch, p.inputs))
        v = V[B.value_off[b]:B.value_off[b + 1]].reshape(k, p.d + 1)
        g = G[B.grad_off[b]:B.grad_off[b + 1]].reshape(k, p.n, p.d + 1)
        assert np.array_equal(v, sv.cpu().numpy()) and np.array_equal(g, sg.cpu().numpy())


def test_tiled_autotune_same_values(torch, tmp_path, monkeypatch):
    """The autotuner on a tiled plan (threads per CTA and CTAs per SM only)."""
    monkeypatch.setenv("PES_AUTOTUNE_CACHE", str(tmp_path / "autotune.txt"))
    k, d = 10, 600
    supp, n, coeff, inputs = case(k, d, 5600, N=5, hi=4)
    C, Z = dev(torch, coeff), dev(torch, inputs)
    v0, g0 = pes.Plan(supp, n, d, k).eval_grad(C, Z)
    plan = pes.Plan(supp, n, d, k, autotune=True)
    v1, g1 = plan.eval_grad(C, Z)
    plan.check()
    assert torch.equal(v0, v1) and torch.equal(g0, g1)
    assert (tmp_path / "autotune.txt").exists()
