"""Parity of the CUDA path (through the C-ABI) with the oracle.

Small cases are compared in full, coefficient by coefficient, against the
oracle.  Full-size configurations are compared on the outputs the oracle can
afford: the first coefficients (a truncated series product only involves the
coefficients up to its own degree, so the oracle at a small degree d' gives the
first d'+1 coefficients of the full-degree result exactly), and on Euler's
identity for homogeneous polynomials at the full degree.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_10881_gb300 import pes, synth
from paper_2101_10881_gb300.synth import KS, random_md
from tests.exact import TOL, exact_ints, normwise_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    pes.build()
    assert _t.cuda.is_available()
    return _t


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(torch, prob, **opts):
    plan = pes.Plan(prob.supports, prob.n, prob.d, prob.k, **opts)
    v, g = plan.eval_grad(dev(torch, prob.coeff), dev(torch, prob.inputs))
    plan.check()
    return v.cpu().numpy(), g.cpu().numpy(), plan


def normalised(a, half_ulp=True):
    """Every coefficient's limbs are nonoverlapping: |x_{l+1}| <= ulp(x_l) / 2
    (series outputs, rounded to nearest limb by limb), or <= ulp(x_l) (the
    renormalised results of md_add / md_mul)."""
    a = np.asarray(a)
    f = 0.5 if half_ulp else 1.0
    for l in range(a.shape[0] - 1):
        hi, lo = a[l], a[l + 1]
        bad = np.where(hi == 0.0, lo != 0.0, np.abs(lo) > np.spacing(np.abs(hi)) * f)
        if bad.any():
            return False
    return True


@pytest.mark.parametrize("k", KS)
def test_md_binary(torch, k):
    rng = np.random.default_rng(k)
    cnt = 257
    x = random_md(rng, k, (cnt,))
    y = random_md(rng, k, (cnt,)) * np.ldexp(1.0, rng.integers(-70, 70, size=cnt))
    add = pes.md_binary("add", dev(torch, x), dev(torch, y)).cpu().numpy()
    mul = pes.md_binary("mul", dev(torch, x), dev(torch, y)).cpu().numpy()
    for i in range(cnt):
        ra = O.md_add(x[:, i], y[:, i])
        rm = O.md_mul(x[:, i], y[:, i])
        assert normwise_err(add[:, i:i + 1], ra[:, None]) <= TOL[k]
        assert normwise_err(mul[:, i:i + 1], rm[:, None]) <= TOL[k]
    assert normalised(add, half_ulp=False) and normalised(mul, half_ulp=False)


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("d", [0, 5, 40])
def test_small_random_polynomials(torch, k, d):
    rng = np.random.default_rng(1000 + 10 * k + d)
    n, N = 7, 12
    supp = synth.random_supports(rng, n, N, 1, 6)
    prob = synth.Problem("small", n, d, k, supp, random_md(rng, k, (N + 1, d + 1)), random_md(rng, k, (n, d + 1)))
    v, g, _ = run(torch, prob)
    vi, gi, _ = run(torch, prob, arith="int")
    rv, rg = O.eval_grad(supp, n, prob.coeff, prob.inputs)
    assert normwise_err(v, rv) <= TOL[k]
    assert normwise_err(g, rg) <= TOL[k]
    # both variants accumulate exactly; they differ only in the digit width that
    # drops the bits far below the k-th limb (24 vs 28 bits)
    assert normwise_err(vi, rv) <= TOL[k] and normwise_err(gi, rg) <= TOL[k]
    assert normwise_err(v, vi) <= TOL[k] and normwise_err(g, gi) <= TOL[k]
    assert normalised(v) and normalised(g)


@pytest.mark.parametrize("k", [2, 3])
def test_degenerate_single_plans(torch, k):
    """A polynomial with no monomial: the value is a_0 limb for limb and the
    gradient is exactly zero; a variable that no monomial holds has an exactly
    zero gradient series; a polynomial of one variable and one monomial of it
    matches the oracle."""
    rng = np.random.default_rng(500 + k)
    d, n = 20, 4
    a0 = random_md(rng, k, (1, d + 1))
    empty = synth.Problem("empty", n, d, k, [], a0, random_md(rng, k, (n, d + 1)))
    v, g, _ = run(torch, empty)
    assert np.array_equal(v, a0[:, 0]) and not g.any()
    supp = [[0, 2], [2]]  # variables 1 and 3 appear in no monomial
    prob = synth.Problem("holes", n, d, k, supp, random_md(rng, k, (3, d + 1)), random_md(rng, k, (n, d + 1)))
    v, g, _ = run(torch, prob)
    assert not g[:, 1].any() and not g[:, 3].any()
    rv, rg = O.eval_grad(supp, n, prob.coeff, prob.inputs)
    assert normwise_err(v, rv) <= TOL[k] and normwise_err(g, rg) <= TOL[k]
    one = synth.Problem("one", 1, d, k, [[0]], random_md(rng, k, (2, d + 1)), random_md(rng, k, (1, d + 1)))
    v, g, _ = run(torch, one)
    rv, rg = O.eval_grad([[0]], 1, one.coeff, one.inputs)
    assert normwise_err(v, rv) <= TOL[k] and normwise_err(g, rg) <= TOL[k]


@pytest.mark.parametrize("threads", [0, 96, 256, 320])
def test_ragged_degree_several_tiles(torch, threads):
    """d = 152: 153 coefficients (a ragged last warp), k = 4, monomials of up to
    5 variables, an unused variable and a one-variable monomial; CTA widths from
    one lane per coefficient pair (96) to four (320)."""
    k, d, n = 4, 152, 6
    supp = [[0, 1, 2, 3, 4], [1, 3], [2], [0, 2, 4], [1, 2, 3, 4]]
    rng = np.random.default_rng(5)
    prob = synth.Problem("ragged", n, d, k, supp, random_md(rng, k, (len(supp) + 1, d + 1)),
                         random_md(rng, k, (n, d + 1)))
    v, g, plan = run(torch, prob, threads=threads)
    rv, rg = O.eval_grad(supp, n, prob.coeff, prob.inputs)
    assert normwise_err(v, rv) <= TOL[k]
    assert normwise_err(g, rg) <= TOL[k]
    assert np.all(g[:, 5] == 0.0)  # x_5 appears nowhere
    info = plan.info()
    assert info["conv_jobs"] == 12 + 3 + 1 + 6 + 9


@pytest.mark.parametrize("k,dmax", [(10, 471), (8, 543), (2, 1351)])
def test_maximum_degree(torch, k, dmax):
    """The largest degree whose whole operand series one job stages in the
    integer variant (both series, their digits and the exchange rows in one
    CTA's shared memory), every output coefficient against the oracle; one
    degree more goes to the tiled kernel, against the oracle too."""
    rng = np.random.default_rng(4000 + k)
    supp, n = [[0, 1], [1, 2, 3]], 4
    for d, tile in ((dmax, 0), (dmax + 1, 128)):
        prob = synth.Problem("dmax", n, d, k, supp, random_md(rng, k, (3, d + 1)), random_md(rng, k, (n, d + 1)))
        v, g, plan = run(torch, prob)
        assert plan.info()["arith_name"] == "int" and plan.info()["tile"] == tile
        rv, rg = O.eval_grad(supp, n, prob.coeff, prob.inputs)
        assert normwise_err(v, rv) <= TOL[k]
        assert normwise_err(g, rg) <= TOL[k]
        assert normalised(v) and normalised(g)


@pytest.mark.parametrize("threads", [96, 192, 256])
def test_staging_depths_agree(torch, threads):
    """Staging depth 2 (the next job claimed, and staged when its operands are
    complete, while the current one is rounded) gives the same bits as depth 1,
    whether the staging thread has no coefficient of its own (threads > d+1) or
    is thread 0; a single long monomial makes consecutive jobs depend on each
    other, so the next job is often not ready when claimed."""
    k, d = 4, 152
    rng = np.random.default_rng(77)
    supp = [list(range(12)), [0, 3, 5], [2, 7], [1, 4, 6, 8, 9, 10, 11]]
    n = 12
    prob = synth.Problem("staging", n, d, k, supp, random_md(rng, k, (len(supp) + 1, d + 1)),
                         random_md(rng, k, (n, d + 1)))
    v1, g1, p1 = run(torch, prob, threads=threads, staging=1)
    v2, g2, p2 = run(torch, prob, threads=threads, staging=2)
    assert p1.info()["staging"] == 1 and p2.info()["staging"] == 2
    assert np.array_equal(v1, v2) and np.array_equal(g1, g2)
    rv, rg = O.eval_grad(supp, n, prob.coeff, prob.inputs)
    assert normwise_err(v2, rv) <= TOL[k]
    assert normwise_err(g2, rg) <= TOL[k]


@pytest.mark.parametrize("split", [2, 4, 8, 16])
def test_split_jobs_agree(torch, split):
    """Jobs split into parts over ranges of coefficient pairs (each part with a
    flag of its own, dependants waiting for all parts) give the same bits as
    whole jobs, forward and VJP, for an odd and an even number of coefficients
    and for a degree with fewer pairs than parts."""
    k = 4
    rng = np.random.default_rng(88 + split)
    supp = [list(range(9)), [0, 3, 5], [2, 7], [1, 4, 6, 8]]
    n = 9
    for d in (152, 41, 2):
        prob = synth.Problem("split", n, d, k, supp, random_md(rng, k, (len(supp) + 1, d + 1)),
                             random_md(rng, k, (n, d + 1)))
        v1, g1, p1 = run(torch, prob, split=1)
        v2, g2, p2 = run(torch, prob, split=split)
        assert p2.info()["split"] == split
        assert np.array_equal(v1, v2) and np.array_equal(g1, g2)
        u = dev(torch, random_md(rng, k, (d + 1,)))
        C, Z = dev(torch, prob.coeff), dev(torch, prob.inputs)
        r1 = p1.vjp(C, Z, u)
        r2 = p2.vjp(C, Z, u)
        p2.check()
        assert all(torch.equal(a, b) for a, b in zip(r1, r2))
    rv, rg = O.eval_grad(supp, n, prob.coeff, prob.inputs)
    assert normwise_err(v2, rv) <= TOL[k] and normwise_err(g2, rg) <= TOL[k]


def max_digit_value(k):
    """A k-double whose 28-bit digits, on the grid of its leading limb, are all
    2^27 - 1 (up to the rounding of the last limb): the largest same-signed digit
    products the integer variant's accumulators can meet."""
    from fractions import Fraction
    nd = (53 * k) // 28 + 1
    f = sum(Fraction(2 ** 27 - 1, 2 ** (28 * p)) for p in range(1, nd + 1))
    return np.array(synth.round_fraction_to_limbs(f, k))


@pytest.mark.parametrize("arith", ["int", "fp64"])
@pytest.mark.parametrize("k", [2, 10])
def test_same_signed_maximal_digits(torch, k, arith):
    """Every input coefficient has all its digits near 2^27 and the same sign, so
    every digit product is close to 2^54 and nothing cancels: the exact digit sums
    of a degree-152 convolution exceed 64 bits unless partial sums are carried
    before they are added up."""
    d, n = 152, 2
    supp = [[0, 1]]
    inputs = np.zeros((k, n, d + 1))
    inputs[:, :, :] = max_digit_value(k)[:, None, None]
    coeff = np.zeros((k, 2, d + 1))
    coeff[0, 1, 0] = 1.0
    prob = synth.Problem("maxdig", n, d, k, supp, coeff, inputs)
    v, g, _ = run(torch, prob, arith=arith)
    rv, rg = O.eval_grad(supp, n, coeff, inputs)
    assert normwise_err(v, rv) <= TOL[k]
    assert normwise_err(g, rg) <= TOL[k]


def test_config0_full(torch):
    """p1 at d=8 in double double, every output coefficient."""
    prob = synth.config0()
    v, g, plan = run(torch, prob)
    rv, rg = O.eval_grad(prob.supports, prob.n, prob.coeff, prob.inputs)
    assert normwise_err(v, rv) <= TOL[2]
    assert normwise_err(g, rg) <= TOL[2]
    assert plan.info()["conv_jobs"] == 16380


def truncated(prob, dd):
    return prob.coeff[:, :, : dd + 1].copy(), prob.inputs[:, :, : dd + 1].copy()


def euler_check(prob, v, g, degree):
    """sum_i z_i * g_i == degree * (v - a_0), exactly in truncated arithmetic."""
    k = prob.k
    lhs = O.conv_many(prob.inputs, g)  # (k, n, d+1)
    (li, vi, ai), _ = exact_ints([lhs, v[:, None, :], prob.coeff[:, :1, :]])
    s = li.sum(axis=0)
    rhs = degree * (vi[0] - ai[0])
    num = max(abs(int(a) - int(b)) for a, b in zip(s, rhs))
    den = max(abs(int(b)) for b in rhs)
    return num / den


def test_config1_full_size(torch):
    """p2-like, n=128, 128 monomials of 64 variables, d=152, deca double."""
    prob = synth.config1()
    v, g, plan = run(torch, prob)
    assert plan.info()["conv_jobs"] == 24192
    dd = 2
    c, z = truncated(prob, dd)
    rv, rg = O.eval_grad(prob.supports, prob.n, c, z)
    assert normwise_err(v[:, : dd + 1], rv) <= TOL[10]
    assert normwise_err(g[:, :, : dd + 1], rg) <= TOL[10]
    assert euler_check(prob, v, g, 64) <= 1e3 * TOL[10]
    assert normalised(v) and normalised(g)


def test_config2_full_size(torch):
    """p3, n=128, all 8128 pairs, d=152, quad double."""
    prob = synth.config2()
    v, g, plan = run(torch, prob)
    dd = 8
    c, z = truncated(prob, dd)
    rv, rg = O.eval_grad(prob.supports, prob.n, c, z)
    assert normwise_err(v[:, : dd + 1], rv) <= TOL[4]
    assert normwise_err(g[:, :, : dd + 1], rg) <= TOL[4]
    assert euler_check(prob, v, g, 2) <= 1e3 * TOL[4]


@pytest.mark.parametrize("k", [1, 2, 4, 10])
def test_vjp_matches_oracle(torch, k):
    rng = np.random.default_rng(300 + k)
    n, N, d = 6, 9, 12
    supp = synth.random_supports(rng, n, N, 1, 5)
    coeff = random_md(rng, k, (N + 1, d + 1))
    inputs = random_md(rng, k, (n, d + 1))
    u = random_md(rng, k, (d + 1,))
    plan = pes.Plan(supp, n, d, k)
    C, Z, U = dev(torch, coeff), dev(torch, inputs), dev(torch, u)
    gi, gc = plan.vjp(C, Z, U, reuse_forward=False)
    plan.eval_grad(C, Z)
    gi2, gc2 = plan.vjp(C, Z, U, reuse_forward=True)
    plan.check()
    ri, rc = O.vjp(supp, n, coeff, inputs, u)
    gi, gc = gi.cpu().numpy(), gc.cpu().numpy()
    assert normwise_err(gi, ri) <= TOL[k]
    assert normwise_err(gc, rc) <= TOL[k]
    assert np.array_equal(gi, gi2.cpu().numpy()) and np.array_equal(gc, gc2.cpu().numpy())


def exact_dot(a, b):
    """Exact sum_j a_j b_j of two limb-major series (k_a, S) and (k_b, S)."""
    from fractions import Fraction
    (ai, bi), e = exact_ints([a, b])
    return Fraction(sum(int(x) * int(y) for x, y in zip(ai, bi))) * Fraction(2) ** (2 * e)


def test_vjp_central_differences_octo(torch):
    """Config 2 shape (pairs of variables) at reduced size: the VJP in quad double
    against central differences of L = <u, v> evaluated in octo double.  L is
    affine in every input series, so the difference quotient is exact up to the
    octo double rounding of v."""
    from fractions import Fraction
    n, d = 24, 40
    supp = synth.supports_p3(n)
    rng = np.random.default_rng(17)
    c8 = random_md(rng, 8, (len(supp) + 1, d + 1))
    z8 = random_md(rng, 8, (n, d + 1))
    u8 = random_md(rng, 8, (d + 1,))
    p4 = pes.Plan(supp, n, d, 4)
    gi, gc = p4.vjp(dev(torch, c8[:4].copy()), dev(torch, z8[:4].copy()), dev(torch, u8[:4].copy()))
    gi, gc = gi.cpu().numpy(), gc.cpu().numpy()
    p8 = pes.Plan(supp, n, d, 8, with_vjp=False)
    h = 2.0 ** -20
    for trial in range(4):
        dirn = np.ldexp(rng.integers(-8, 9, size=d + 1).astype(float), -3)
        for which in ("input", "coeff"):
            idx = int(rng.integers(0, n if which == "input" else len(supp) + 1))
            cp, cm, zp, zm = c8.copy(), c8.copy(), z8.copy(), z8.copy()
            if which == "input":
                zp[0, idx] += h * dirn
                zm[0, idx] -= h * dirn
                grad = gi[:, idx]
            else:
                cp[0, idx] += h * dirn
                cm[0, idx] -= h * dirn
                grad = gc[:, idx]
            vp = p8.eval_grad(dev(torch, cp), dev(torch, zp))[0].cpu().numpy()
            vm = p8.eval_grad(dev(torch, cm), dev(torch, zm))[0].cpu().numpy()
            fd = (exact_dot(vp, u8) - exact_dot(vm, u8)) / (2 * Fraction(h))
            an = exact_dot(grad, dirn[None, :])
            scale = exact_dot(np.abs(grad), np.abs(dirn)[None, :])
            assert abs(fd - an) <= scale * Fraction(1, 10 ** 55)


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_matches_single_plans(torch, autotune, tmp_path, monkeypatch):
    """Mixed degrees (several CTA-shape groups on forked streams in one graph),
    with and without the autotuner: every instance equals its own plan bit for
    bit and the oracle within tolerance."""
    monkeypatch.setenv("PES_AUTOTUNE_CACHE", str(tmp_path / "autotune.txt"))
    rng = np.random.default_rng(40)
    k = 2
    insts, probs = [], []
    for b, d in enumerate([0, 7, 15, 31, 40, 63, 100, 152]):
        n = int(rng.integers(3, 9))
        N = int(rng.integers(1, 15))
        supp = synth.random_supports(rng, n, N, 1, min(n, 5))
        probs.append(synth.Problem(f"b{b}", n, d, k, supp, random_md(rng, k, (N + 1, d + 1)),
                                   random_md(rng, k, (n, d + 1))))
        insts.append((supp, n, d))
    B = pes.Batch(insts, k, autotune=autotune)
    assert B.info()["grid"] >= 4  # groups of CTA shapes 32, 64, 128, 160
    C = dev(torch, np.concatenate([p.coeff.ravel() for p in probs]))
    Z = dev(torch, np.concatenate([p.inputs.ravel() for p in probs]))
    ln = B.lengths()
    V = torch.empty(ln["value"], dtype=torch.float64, device="cuda")
    G = torch.empty(ln["grad"], dtype=torch.float64, device="cuda")
    for _ in range(2):  # second call replays the captured graph
        B.eval_grad(C, Z, V, G)
    B.check()
    V, G = V.cpu().numpy(), G.cpu().numpy()
    for b, p in enumerate(probs):
        v = V[B.value_off[b]:B.value_off[b + 1]].reshape(k, p.d + 1)
        g = G[B.grad_off[b]:B.grad_off[b + 1]].reshape(k, p.n, p.d + 1)
        sv, sg, _ = run(torch, p)
        assert np.array_equal(v, sv) and np.array_equal(g, sg)
        rv, rg = O.eval_grad(p.supports, p.n, p.coeff, p.inputs)
        assert normwise_err(v, rv) <= TOL[k] and normwise_err(g, rg) <= TOL[k]
    if autotune:
        assert (tmp_path / "autotune.txt").exists()


def test_plan_autotune_same_values(torch, tmp_path, monkeypatch):
    """The first call of an autotuned plan times several CTA shapes on the
    caller's data; the values equal those of the default shape, and the choice
    is cached."""
    monkeypatch.setenv("PES_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    k, d = 10, 100
    rng = np.random.default_rng(123)
    supp = synth.random_supports(rng, 12, 20, 2, 6)
    prob = synth.Problem("tune", 12, d, k, supp, random_md(rng, k, (21, d + 1)), random_md(rng, k, (12, d + 1)))
    v0, g0, _ = run(torch, prob)
    v1, g1, plan = run(torch, prob, autotune=True)
    assert np.array_equal(v0, v1) and np.array_equal(g0, g1)
    gi, gc = plan.vjp(dev(torch, prob.coeff), dev(torch, prob.inputs), dev(torch, random_md(rng, k, (d + 1,))))
    plan.check()
    assert (tmp_path / "tune.txt").read_text().strip()


def test_later_small_plan_keeps_large_plan_launchable(torch):
    """The shared-memory limit is per kernel function: building a plan for a small
    degree after one for a large degree must not break the large one."""
    k = 4
    rng = np.random.default_rng(9)
    big = synth.Problem("big", 5, 152, k, [[0, 1, 2], [1, 3, 4]], random_md(rng, k, (3, 153)),
                        random_md(rng, k, (5, 153)))
    plan_big = pes.Plan(big.supports, big.n, big.d, k)
    pes.Plan([[0, 1]], 2, 3, k)  # small degree, built afterwards
    v, g = plan_big.eval_grad(dev(torch, big.coeff), dev(torch, big.inputs))
    plan_big.check()
    rv, rg = O.eval_grad(big.supports, big.n, big.coeff, big.inputs)
    assert normwise_err(v.cpu().numpy(), rv) <= TOL[k] and normwise_err(g.cpu().numpy(), rg) <= TOL[k]


def test_bounded_wait_reports_timeout(torch):
    """A job that waits on a flag nobody sets gives up after the bound and
    reports PES_ETIMEOUT; the context stays usable."""
    assert pes.selftest_timeout(300) == "PES_ETIMEOUT"
    prob = synth.config0()
    v, g, _ = run(torch, prob)
    rv = O.eval_grad(prob.supports, prob.n, prob.coeff, prob.inputs, grad=False)
    assert normwise_err(v, rv) <= TOL[2]


def test_invalid_arguments(torch):
    with pytest.raises(pes.PesError) as e:
        pes.Plan([[0, 1]], 2, 4, 6)
    assert e.value.code == 2
    with pytest.raises(pes.PesError) as e:
        pes.Plan([[1, 0]], 2, 4, 2)
    assert e.value.code == 1
    with pytest.raises(pes.PesError) as e:
        pes.Plan([[0]], 1, 16384, 2)  # above the largest degree
    assert e.value.code == 7
    with pytest.raises(pes.PesError) as e:
        pes.Plan([[0, 1]], 2, 900, 10, tile=512)  # 256 pairs per tile: more than 256 lanes at k=10
    assert e.value.code == 7
    for bad in (12, 20, 2048):
        with pytest.raises(pes.PesError) as e:
            pes.Plan([[0, 1]], 2, 40, 2, tile=bad)
        assert e.value.code == 1
    for bad in (3, 32, -1):
        with pytest.raises(pes.PesError) as e:
            pes.Plan([[0, 1]], 2, 40, 2, split=bad)
        assert e.value.code == 1
