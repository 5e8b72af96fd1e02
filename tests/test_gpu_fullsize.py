"""Parity at the full sizes of the headline workloads, in the launch
configuration the benchmark times (autotuned CTA shape).

  * p2-like shape (n=128, 128 monomials of 64 variables, d=152, deca double)
    with exp-series inputs and degree-0 coefficients: every coefficient of the
    value and of all 128 gradient series against the exact closed form;
  * the same workload on its random series: two whole gradient series at the
    full degree against the oracle;
  * p3 (n=128, all 8128 pairs, d=152, quad double): the VJP of an upstream
    series with respect to all inputs and all 8129 coefficient series against
    exact central differences of <u, v> evaluated in octo double, and sampled
    coefficient gradients against the oracle element by element;
  * the batched recipe (2048 instances, double double): 16 sampled instances
    against the oracle element by element.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_10881_gb300 import pes, synth
from paper_2101_10881_gb300.synth import random_md
from tests.exact import TOL, exact_ints, exp_series_fixed, limbs_fixed, normwise_err, normwise_err_ints

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    pes.build()
    assert _t.cuda.is_available()
    return _t


@pytest.fixture()
def tune_cache(tmp_path, monkeypatch):
    monkeypatch.setenv("PES_AUTOTUNE_CACHE", str(tmp_path / "autotune.txt"))


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def eval_tuned(torch, prob):
    """eval+grad with the autotuned plan (as the benchmark runs it) and with the
    default launch shape; both give the same bits (exact sums rounded once)."""
    C, Z = dev(torch, prob.coeff), dev(torch, prob.inputs)
    tuned = pes.Plan(prob.supports, prob.n, prob.d, prob.k, with_vjp=False, autotune=True)
    v, g = tuned.eval_grad(C, Z)
    v, g = tuned.eval_grad(C, Z)  # after the tuning call
    tuned.check()
    plain = pes.Plan(prob.supports, prob.n, prob.d, prob.k, with_vjp=False)
    v0, g0 = plain.eval_grad(C, Z)
    plain.check()
    assert torch.equal(v, v0) and torch.equal(g, g0)
    return v.cpu().numpy(), g.cpu().numpy(), tuned.info()


def test_config1_shape_closed_form_every_coefficient(torch, tune_cache):
    """Inputs z_i = exp(a_i t) with a_i = A_i / 2^20, A_i uniform in [0, 2^20],
    degree-0 coefficients c_m (random deca double scalars of both signs).  Then
    v_j = c_0 [j = 0] + sum_m c_m s_m^j / j! with s_m the sum of a_i over S_m,
    and (d p / d x_i)_j = sum_{m : i in S_m} c_m (s_m - a_i)^j / j!, evaluated
    exactly in integers at scale 2^-1600.  The inputs are rounded to 10 limbs
    (relative error below 2^-529 per coefficient); with a_i >= 0 every product
    series has positive coefficients, so that rounding moves every product
    coefficient by at most 64 * 2^-529 of itself, far inside the tolerance
    (1e-150, about 2^-498) after the cancellation between monomials."""
    k, d, n = 10, 152, 128
    supports = synth.supports_p2()
    rng = np.random.default_rng(1)
    A = [int(a) for a in rng.integers(0, 2 ** 20 + 1, size=n)]
    avals = [a / 2 ** 20 for a in A]
    inputs = synth.exp_inputs(avals, d, k)
    coeff = synth.scalar_coeffs(rng, k, len(supports), d)
    prob = synth.Problem("p2 exp", n, d, k, supports, coeff, inputs)
    v, g, info = eval_tuned(torch, prob)
    assert info["conv_jobs"] == 24192 and info["arith_name"] == "int"

    F = 1600
    cs = [sum((Fraction(float(x)) for x in coeff[:, m, 0]), Fraction(0)) for m in range(len(supports) + 1)]
    S = [sum(A[i] for i in s) for s in supports]
    ref_v = [0] * (d + 1)
    ref_v[0] += cs[0].numerator * (1 << F) // cs[0].denominator
    ref_g = [[0] * (d + 1) for _ in range(n)]
    for m, s in enumerate(supports):
        for j, t in enumerate(exp_series_fixed(cs[m + 1], S[m], 20, d, F)):
            ref_v[j] += t
        for i in s:
            row = ref_g[i]
            for j, t in enumerate(exp_series_fixed(cs[m + 1], S[m] - A[i], 20, d, F)):
                row[j] += t
    gv = limbs_fixed(v, F)
    gg = limbs_fixed(g, F)
    assert normwise_err_ints(gv, ref_v) <= TOL[k]
    worst = max(normwise_err_ints(gg[i], ref_g[i]) for i in range(n))
    assert worst <= TOL[k], worst


def test_config1_random_two_gradient_series_full_degree(torch, tune_cache):
    """The random deca double series of the workload: the gradient series of the
    two variables that occur in the fewest monomials (50 and 51 of 128), every
    coefficient up to d = 152, against the oracle.  The partial with respect to
    x_i is the value of sum_{m : i in S_m} a_m prod_{j in S_m, j != i} x_j,
    which the oracle evaluates naively (63 products per monomial, each rounded
    to 10 limbs, the sum exact and rounded once)."""
    prob = synth.config1()
    v, g, info = eval_tuned(torch, prob)
    counts = np.zeros(prob.n, dtype=int)
    for s in prob.supports:
        counts[s] += 1
    for i in (int(x) for x in np.argsort(counts, kind="stable")[:2]):
        rows = [m for m, s in enumerate(prob.supports) if i in s]
        supp_i = [[v_ for v_ in prob.supports[m] if v_ != i] for m in rows]
        coeff_i = np.zeros((prob.k, len(rows) + 1, prob.d + 1))
        coeff_i[:, 1:] = prob.coeff[:, [m + 1 for m in rows]]
        ref = O.eval_grad(supp_i, prob.n, coeff_i, prob.inputs, grad=False)
        assert normwise_err(g[:, i], ref) <= TOL[prob.k], i


def two_sum_limbs(base, delta, k_out):
    """base (k, ...) limbs plus one double delta per coefficient, exactly, as
    k_out >= k + 1 limbs: the leading limb and delta by TwoSum (sum and its
    exact error), then the other limbs of base, then zero limbs.  Every lower
    limb stays far below the leading one (delta is at most 2^-20)."""
    a = base[0]
    s = a + delta
    bb = s - a
    e = (a - (s - bb)) + (delta - bb)
    out = np.zeros((k_out,) + base.shape[1:])
    out[0] = s
    out[1] = e
    out[2:base.shape[0] + 1] = base[1:]
    return out


def exact_dot_ints(gi, wi):
    return sum(int(a) * int(b) for a, b in zip(gi.ravel(), wi.ravel()))


def test_config2_full_size_vjp_central_differences(torch):
    """p3 at d=152: the quad double VJP of a random upstream series u with respect
    to all 128 input series and all 8129 coefficient series.  Along random
    directions w (dense over all inputs, or over all coefficient series), the
    directional derivative <VJP, w> is compared with (L(+h) - L(-h)) / 2h,
    L(t) = <u, v(x + t w)> with v evaluated in octo double (h = 2^-20).  v is
    quadratic along an input direction and linear along a coefficient
    direction, so the central difference is exact up to the octo double
    rounding of v.  The bound is the quad double tolerance applied per series
    (each series within 1e-60 of its largest coefficient) plus the octo double
    evaluation error divided by 2h."""
    prob = synth.config2()
    k, d, n, N = prob.k, prob.d, prob.n, prob.N
    rng = np.random.default_rng(99)
    u = random_md(rng, k, (d + 1,))
    C4, Z4, U = dev(torch, prob.coeff), dev(torch, prob.inputs), dev(torch, u)
    p4 = pes.Plan(prob.supports, n, d, k)
    p4.eval_grad(C4, Z4)
    gi, gc = p4.vjp(C4, Z4, U, reuse_forward=True)
    gi2, gc2 = p4.vjp(C4, Z4, U, reuse_forward=False)
    p4.check()
    assert torch.equal(gi, gi2) and torch.equal(gc, gc2)
    gi, gc = gi.cpu().numpy(), gc.cpu().numpy()

    # sampled coefficient gradients element by element: grad_coeff[m] is the
    # correlation of u with the monomial product z_i z_j
    for m in (int(x) for x in rng.choice(N, size=8, replace=False)):
        i, j = prob.supports[m]
        mono = O.conv(prob.inputs[:, i], prob.inputs[:, j])
        assert normwise_err(gc[:, m + 1], O.corr(u, mono)) <= TOL[k]
    assert np.array_equal(gc[:, 0], u)

    p8 = pes.Plan(prob.supports, n, d, 8, with_vjp=False)
    c8 = np.zeros((8, N + 1, d + 1))
    c8[:k] = prob.coeff
    z8 = np.zeros((8, n, d + 1))
    z8[:k] = prob.inputs
    h_exp = 20
    h = Fraction(1, 2 ** h_exp)
    (ui,), ue = exact_ints([u])
    u_abs = float(np.abs(u[0]).sum()) * 1.01

    def loss(c, z):
        v = p8.eval_grad(dev(torch, c), dev(torch, z))[0].cpu().numpy()
        (vi,), ve = exact_ints([v])
        return Fraction(sum(int(a) * int(b) for a, b in zip(vi, ui))) * Fraction(2) ** (ve + ue), \
            float(np.abs(v[0]).max())

    (gci,), gce = exact_ints([gc])
    (gii,), gie = exact_ints([gi])
    for which in ("input", "coeff"):
        grad, gint, gexp = (gi, gii, gie) if which == "input" else (gc, gci, gce)
        per_series_max = np.abs(grad[0]).max(axis=-1) * 1.01
        for trial in range(4):
            w = np.ldexp(rng.integers(-8, 9, size=grad.shape[1:]).astype(float), -3)
            delta = np.ldexp(w, -h_exp)
            if which == "input":
                lp, vmax_p = loss(c8, two_sum_limbs(prob.inputs, delta, 8))
                lm, vmax_m = loss(c8, two_sum_limbs(prob.inputs, -delta, 8))
            else:
                lp, vmax_p = loss(two_sum_limbs(prob.coeff, delta, 8), z8)
                lm, vmax_m = loss(two_sum_limbs(prob.coeff, -delta, 8), z8)
            fd = (lp - lm) / (2 * h)
            an = Fraction(exact_dot_ints(gint, np.ldexp(w, 3).astype(np.int64))) * Fraction(2) ** (gexp - 3)
            # |L error| <= TOL[8] max|v| sum|u| at each end, divided by 2h; doubled for safety
            bound = (TOL[k] * float((per_series_max * np.abs(w).sum(axis=-1)).sum())
                     + 2 * TOL[8] * max(vmax_p, vmax_m) * u_abs * 2 ** h_exp)
            assert abs(float(fd - an)) <= bound, (which, trial, float(fd - an), bound)


def test_config3_batch_sampled_instances(torch, tune_cache):
    """The whole batched recipe (2048 instances: n uniform in 8-128, 16-2048
    monomials of 2-8 variables, d from {15, 31, 63, 127, 152}, double double)
    in one autotuned, graph-captured call, as the benchmark runs it; 16
    instances drawn at random (seeded) compared with the oracle element by
    element, twice (the second call replays the graph)."""
    k = 2
    shapes = synth.config3_shapes(seed=0, count=2048)
    rng = np.random.default_rng(7)
    probs = []
    for b, (n, supp, d) in enumerate(shapes):
        N = len(supp)
        probs.append(synth.Problem(f"b{b}", n, d, k, supp, random_md(rng, k, (N + 1, d + 1)),
                                   random_md(rng, k, (n, d + 1))))
    B = pes.Batch([(p.supports, p.n, p.d) for p in probs], k, autotune=True)
    C = dev(torch, np.concatenate([p.coeff.ravel() for p in probs]))
    Z = dev(torch, np.concatenate([p.inputs.ravel() for p in probs]))
    ln = B.lengths()
    V = torch.empty(ln["value"], dtype=torch.float64, device="cuda")
    G = torch.empty(ln["grad"], dtype=torch.float64, device="cuda")
    B.eval_grad(C, Z, V, G)
    first = (V.clone(), G.clone())
    B.eval_grad(C, Z, V, G)
    B.check()
    assert torch.equal(first[0], V) and torch.equal(first[1], G)
    del C, Z, first
    V, G = V.cpu().numpy(), G.cpu().numpy()
    pick = sorted(int(b) for b in np.random.default_rng(2048).choice(len(probs), size=16, replace=False))
    for b in pick:
        p = probs[b]
        v = V[B.value_off[b]:B.value_off[b + 1]].reshape(k, p.d + 1)
        g = G[B.grad_off[b]:B.grad_off[b + 1]].reshape(k, p.n, p.d + 1)
        rv, rg = O.eval_grad(p.supports, p.n, p.coeff, p.inputs)
        assert normwise_err(v, rv) <= TOL[k], b
        assert normwise_err(g, rg) <= TOL[k], b
