"""Job compiler (host, integer only) against the counts the paper prints and a
symbolic interpretation of its job tables.  No GPU needed: these functions of
libpes do not touch the device."""
from collections import Counter

import numpy as np
import pytest

from paper_2101_10881_gb300 import pes, synth
from tests.golden.load import paper_counts

PC = paper_counts()
EXAMPLE = [[0, 2, 5], [0, 1, 4, 5], [1, 2, 3]]  # a1 x1 x3 x6 + a2 x1 x2 x5 x6 + a3 x2 x3 x4


@pytest.fixture(scope="module", autouse=True)
def built():
    pes.build()


def test_example_triplet_and_pair_offsets():
    jobs = pes.jobc_jobs(EXAMPLE, 6, paper_layout=True)
    # f_{1,1} := a_1 * z_1 is the first job of layer 1
    assert list(jobs[0][:3]) == PC["example_triplet_f11"]
    # f_{1,3} is slot 12: the output of the job f_{1,3} := f_{1,2} * z_6
    outs = {tuple(j[:2]): j[2] for j in jobs}
    assert outs[(11, 1 + 3 + 5)] == PC["example_pair_f13"][1]
    st = pes.jobc_stats(EXAMPLE, 6, paper_layout=True)
    assert st["slots"] == PC["example_data_array_series"]


def test_example_layers():
    st = pes.jobc_stats(EXAMPLE, 6)
    assert st["conv_jobs"] == PC["example_convolutions"]
    assert st["layer_sizes"] == PC["example_layers"]


def test_p1_counts():
    supp = synth.supports_p1()
    st = pes.jobc_stats(supp, 16)
    assert st["conv_jobs"] == PC["p1_convolutions"]
    assert st["layer_sizes"] == PC["p1_conv_layers"]
    assert st["paper_add_jobs"] == PC["p1_additions"]
    assert pes.jobc_add_levels(supp, 16) == PC["p1_add_levels"]


def test_p2_layers():
    supp = synth.supports_p2()
    st = pes.jobc_stats(supp, 128)
    assert st["conv_jobs"] == PC["p2_convolutions"]
    assert st["layer_sizes"][:31] == [PC["p2_first_31_layers"]] * 31
    assert st["layers"] == 64


def test_p3_counts():
    supp = synth.supports_p3()
    st = pes.jobc_stats(supp, 128)
    assert st["paper_add_jobs"] == PC["p3_additions"]
    # three products per monomial of two variables (the table's 24,256 is not 3 x 8128)
    assert st["conv_jobs"] == 3 * 8128
    assert st["layer_sizes"] == [2 * 8128, 8128]


@pytest.mark.parametrize("seed", range(4))
def test_data_array_count_formula(seed):
    """Eq. (eqcountnum): 1 + N + n + sum (n_k + max(1, n_k-2) + max(0, n_k-2))."""
    rng = np.random.default_rng(seed)
    n = 12
    supp = synth.random_supports(rng, n, 30, 1, 9)
    st = pes.jobc_stats(supp, n, paper_layout=True)
    expect = 1 + len(supp) + n + sum(len(s) + max(1, len(s) - 2) + max(0, len(s) - 2) for s in supp)
    assert st["slots"] == expect


def symbolic(supports, n, paper_layout=False, exponents=None):
    """Interpret the job table on multisets of symbols; check the schedule."""
    N = len(supports)
    jobs = pes.jobc_jobs(supports, n, paper_layout, exponents=exponents)
    content = {0: Counter(["a0"])}
    for m in range(1, N + 1):
        content[m] = Counter([f"a{m}"])
    for i in range(n):
        content[1 + N + i] = Counter([f"z{i}"])
    ready = {s: 0 for s in content}
    written_in_layer = {}
    for in1, in2, out, layer in jobs:
        assert in1 in content and in2 in content, "operand read before it is produced"
        assert ready[in1] < layer and ready[in2] < layer, "operand produced in the same or a later layer"
        assert (out, layer) not in written_in_layer, "two jobs of one layer write one slot"
        written_in_layer[(out, layer)] = True
        assert layer == 1 + max(ready[in1], ready[in2]), "job not in its earliest layer"
        content[out] = content[in1] + content[in2]
        ready[out] = layer
    return content


@pytest.mark.parametrize("seed", range(6))
def test_symbolic_value_and_gradient(seed):
    rng = np.random.default_rng(100 + seed)
    n = 10
    supp = synth.random_supports(rng, n, 25, 1, 9)
    content = symbolic(supp, n)
    add_ptr, add_src = pes.jobc_add_terms(supp, n)
    N = len(supp)

    def terms(o):
        return sorted(tuple(sorted(content[s].elements())) for s in add_src[add_ptr[o]:add_ptr[o + 1]])

    want_value = sorted([("a0",)] + [tuple(sorted([f"a{m + 1}"] + [f"z{v}" for v in s])) for m, s in enumerate(supp)])
    assert terms(0) == want_value
    for i in range(n):
        want = sorted(tuple(sorted([f"a{m + 1}"] + [f"z{v}" for v in s if v != i]))
                      for m, s in enumerate(supp) if i in s)
        assert terms(1 + i) == want


def test_symbolic_example_paper_layout():
    symbolic(EXAMPLE, 6, paper_layout=True)


def test_invalid_supports():
    for bad, n in (([[1, 0]], 3), ([[0, 0]], 3), ([[3]], 3), ([[]], 3), ([[0]], 0)):
        with pytest.raises(pes.PesError) as e:
            pes.jobc_stats(bad, n)
        assert e.value.code == 1


def test_flop_metric_reproduces_paper():
    """Sec. 6.2: the P100 figure of 1.25 TFLOPS counts (d+1)^2 deca double
    multiplications and d(d+1) additions per convolution plus d+1 per addition."""
    mul, add = pes.md_costs(10)
    d = 152
    conv, adds = PC["p1_convolutions"], PC["p1_additions"]
    mul_ops = conv * (d + 1) ** 2 * mul
    add_ops = (conv * d * (d + 1) + adds * (d + 1)) * add
    assert mul_ops == PC["p1_paper_mul_ops_d152"]
    assert add_ops == PC["p1_paper_add_ops_d152"]
    assert mul_ops + add_ops == PC["p1_paper_total_ops_d152"]


def test_bench_paper_convention_count():
    """bench.py's paper-convention count is the same rule: it reproduces the
    paper's total for p1 at d = 152."""
    import bench
    assert bench.paper_convention_ops(PC["p1_convolutions"], PC["p1_additions"], 152, 10) == \
        PC["p1_paper_total_ops_d152"]


@pytest.mark.parametrize("seed", range(4))
def test_symbolic_powers(seed):
    """Monomials with powers (Sec. 3): the value term of monomial m is the
    multiset a_m z_v^{e_v}, the term of the partial for x_i is
    a_m z_i^{e_i - 1} prod_{v != i} z_v^{e_v} with the integer factor e_i, and the
    schedule puts every job in its earliest layer after its operands."""
    rng = np.random.default_rng(300 + seed)
    n = 7
    supp = synth.random_supports(rng, n, 12, 1, 5)
    ex = [[int(e) for e in rng.integers(1, 5, size=len(s_))] for s_ in supp]
    content = symbolic(supp, n, exponents=ex)
    add_ptr, add_src, add_mult = pes.jobc_add_terms(supp, n, exponents=ex)

    def terms(o):
        return sorted((tuple(sorted(content[s_].elements())), int(mu))
                      for s_, mu in zip(add_src[add_ptr[o]:add_ptr[o + 1]], add_mult[add_ptr[o]:add_ptr[o + 1]]))

    def mono(m, skip=None):
        out = [f"a{m + 1}"]
        for v, e in zip(supp[m], ex[m]):
            out += [f"z{v}"] * (e - (1 if v == skip else 0))
        return tuple(sorted(out))

    assert terms(0) == sorted([(("a0",), 1)] + [(mono(m), 1) for m in range(len(supp))])
    for i in range(n):
        want = sorted((mono(m, i), e) for m in range(len(supp)) for v, e in zip(supp[m], ex[m]) if v == i)
        assert terms(1 + i) == want


def test_powers_job_counts():
    """x0^3 x1^2 x2: powers z0^2 (1 job); the common factor z0^2 z1 (1 job);
    a' = a F (1 job); then the 3n - 3 = 6 products of the exponent-one monomial."""
    st = pes.jobc_stats([[0, 1, 2]], 3, exponents=[[3, 2, 1]])
    assert st["conv_jobs"] == 1 + 1 + 1 + 6
    # exponents all 1: exactly the plain tables
    plain = pes.jobc_stats([[0, 1, 2]], 3)
    ones = pes.jobc_stats([[0, 1, 2]], 3, exponents=[[1, 1, 1]])
    assert plain == ones


def test_invalid_exponents():
    for bad in ([[0, 1]], [[1, 65]], [[-1, 2]]):
        with pytest.raises(pes.PesError) as e:
            pes.jobc_stats([[0, 1]], 2, exponents=bad)
        assert e.value.code == 1
    with pytest.raises(pes.PesError):
        pes.jobc_stats([[0, 1]], 2, paper_layout=True, exponents=[[2, 1]])


@pytest.mark.parametrize("powers", [False, True])
@pytest.mark.parametrize("seed", range(3))
def test_symbolic_system(seed, powers):
    """Systems (one job table for P polynomials): output p is polynomial p's
    constant plus its monomials' value terms, output P + p*n + i its partial
    for x_i with the exponent as integer factor, and no term of one
    polynomial lands in another's outputs."""
    rng = np.random.default_rng(500 + seed)
    n, P = 6, 4
    polys = [synth.random_supports(rng, n, int(rng.integers(0, 6)), 1, 4) for _ in range(P)]
    exps = [[[int(e) for e in rng.integers(1, 4, size=len(s_))] for s_ in p_] for p_ in polys] if powers else None
    supp = [m for p_ in polys for m in p_]
    flat_ex = [e for pe in exps for e in pe] if powers else None
    N = len(supp)
    content = symbolic(supp, n, exponents=flat_ex) if N else {}
    const0, add_ptr, add_src, add_mult = pes.jobc_add_terms_system(polys, n, exponents=exps)
    for p in range(P):
        content[const0 + p] = Counter([f"c{p}"])

    def terms(o):
        return sorted((tuple(sorted(content[s_].elements())), int(mu))
                      for s_, mu in zip(add_src[add_ptr[o]:add_ptr[o + 1]], add_mult[add_ptr[o]:add_ptr[o + 1]]))

    m0 = 0
    for p, p_ in enumerate(polys):
        def mono(m, skip=None):
            out = [f"a{m0 + m + 1}"]
            for t, v in enumerate(p_[m]):
                e = exps[p][m][t] if powers else 1
                out += [f"z{v}"] * (e - (1 if v == skip else 0))
            return tuple(sorted(out))

        assert terms(p) == sorted([((f"c{p}",), 1)] + [(mono(m), 1) for m in range(len(p_))])
        for i in range(n):
            want = sorted((mono(m, i), exps[p][m][t] if powers else 1)
                          for m in range(len(p_)) for t, v in enumerate(p_[m]) if v == i)
            assert terms(P + p * n + i) == want
        m0 += len(p_)
