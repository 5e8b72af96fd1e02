"""Seeded synthetic inputs shaped like the paper's test polynomials.

This module holds input generation only: supports, random multiple double
series and the exp-series inputs with a closed form.  It contains none of the
evaluation arithmetic, so the CUDA path and the oracle can both be fed from it.

Shapes (Verschelde 2021, Sec. 6.1 "Equipment and Test Polynomials", Table
tabtestpols):
  * p1: n=16, all C(16,4)=1820 products of four distinct variables;
  * p2-like: n=128, 128 monomials, each a uniformly drawn 64-subset;
  * p3: n=128, all 8128 products x_i x_j with i<j.
Every coefficient a_k and input z_i is a full random series: limb 0 uniform in
[-1,1]; limb l (l >= 1) uniform in (-1,1) times half an ulp of limb l-1, so that
the limbs never overlap and no renormalisation is needed.

Layouts: coefficient series (k, N+1, d+1) with index 0 the constant term a_0;
input series (k, n, d+1); supports are lists of increasing 0-based indices.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

KS = (1, 2, 3, 4, 5, 8, 10)


def random_md(rng: np.random.Generator, k: int, shape) -> np.ndarray:
    """Random normalised k-limb numbers, float64 array of shape (k, *shape)."""
    shape = tuple(np.atleast_1d(shape)) if not isinstance(shape, tuple) else shape
    out = np.empty((k,) + shape)
    out[0] = rng.uniform(-1.0, 1.0, size=shape)
    for l in range(1, k):
        half_ulp = np.spacing(np.abs(out[l - 1])) * 0.5
        half_ulp = np.where(out[l - 1] == 0.0, 0.0, half_ulp)
        out[l] = rng.uniform(-1.0, 1.0, size=shape) * half_ulp
    return out


@dataclass
class Problem:
    """One polynomial with its coefficient and input series."""
    name: str
    n: int
    d: int
    k: int
    supports: list
    coeff: np.ndarray = field(repr=False)   # (k, N+1, d+1)
    inputs: np.ndarray = field(repr=False)  # (k, n, d+1)

    @property
    def N(self) -> int:
        return len(self.supports)

    def csr(self):
        ptr = np.zeros(self.N + 1, dtype=np.int32)
        idx = []
        for m, s in enumerate(self.supports):
            idx.extend(int(v) for v in s)
            ptr[m + 1] = len(idx)
        return ptr, np.asarray(idx, dtype=np.int32)


def supports_p1(n: int = 16, m: int = 4):
    return [list(c) for c in itertools.combinations(range(n), m)]


def supports_p2(n: int = 128, N: int = 128, m: int = 64, seed: int = 0):
    rng = np.random.default_rng(seed)
    return [sorted(int(v) for v in rng.choice(n, size=m, replace=False)) for _ in range(N)]


def supports_p3(n: int = 128):
    return [[i, j] for i in range(n) for j in range(i + 1, n)]


def random_supports(rng, n: int, N: int, lo: int, hi: int):
    """N monomials, each of a uniform number in [lo, hi] of distinct variables."""
    out = []
    for _ in range(N):
        nk = int(rng.integers(lo, min(hi, n) + 1))
        out.append(sorted(int(v) for v in rng.choice(n, size=nk, replace=False)))
    return out


def make_problem(name, supports, n, d, k, seed=0) -> Problem:
    rng = np.random.default_rng(seed)
    N = len(supports)
    coeff = random_md(rng, k, (N + 1, d + 1))
    inputs = random_md(rng, k, (n, d + 1))
    return Problem(name, n, d, k, supports, coeff, inputs)


def config0(seed: int = 0) -> Problem:
    """p1 at d=8 in double double."""
    return make_problem("p1 n=16 N=1820 m=4 d=8 k=2", supports_p1(), 16, 8, 2, seed)


def config1(seed: int = 0, d: int = 152, k: int = 10) -> Problem:
    """p2-like at d=152 in deca double."""
    return make_problem(f"p2 n=128 N=128 m=64 d={d} k={k}", supports_p2(seed=seed), 128, d, k, seed)


def config2(seed: int = 0, d: int = 152, k: int = 4) -> Problem:
    """p3 at d=152 in quad double."""
    return make_problem(f"p3 n=128 N=8128 m=2 d={d} k={k}", supports_p3(), 128, d, k, seed)


def config3_shapes(seed: int = 0, count: int = 2048):
    """Shapes of the batched workload: list of (n, supports, d)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(8, 129))
        N = int(rng.integers(16, 2049))
        d = int(rng.choice([15, 31, 63, 127, 152]))
        out.append((n, random_supports(rng, n, N, 2, 8), d))
    return out


def small_batch_shapes(seed: int = 0, count: int = 2048):
    """Shapes of a batch of small instances (list of (n, supports, d)): n uniform
    in 4-16, 4-32 monomials of 2-4 distinct variables, d drawn from {7, 15, 31}.
    The batched recipe's own instances are large (thousands of convolutions
    each); these are the instances where one launch per instance is dominated by
    launch and dependency latency."""
    rng = np.random.default_rng(seed + 4242)
    out = []
    for _ in range(count):
        n = int(rng.integers(4, 17))
        N = int(rng.integers(4, 33))
        d = int(rng.choice([7, 15, 31]))
        out.append((n, random_supports(rng, n, N, 2, min(4, n)), d))
    return out


def config3(seed: int = 0, count: int = 2048, k: int = 2):
    probs = []
    for b, (n, supp, d) in enumerate(config3_shapes(seed, count)):
        probs.append(make_problem(f"batch[{b}]", supp, n, d, k, seed + 1 + b))
    return probs


# ---------------------------------------------------------------------------
# exp-series inputs with a closed form
# ---------------------------------------------------------------------------

def round_fraction_to_limbs(f: Fraction, k: int):
    """Nearest-double limbs of an exact rational: limb l = float(remainder)."""
    limbs = []
    r = f
    for _ in range(k):
        x = float(r)
        limbs.append(x)
        r -= Fraction(x)
    return limbs


def exp_series_exact(a: float, d: int):
    """Exact coefficients a^j / j! of exp(a t), j = 0..d, with a taken exactly."""
    fa = Fraction(a)
    out = [Fraction(1)]
    for j in range(1, d + 1):
        out.append(out[-1] * fa / j)
    return out


def exp_inputs(avals, d: int, k: int) -> np.ndarray:
    """(k, n, d+1) limbs of z_i = exp(a_i t) truncated at degree d."""
    n = len(avals)
    out = np.zeros((k, n, d + 1))
    for i, a in enumerate(avals):
        for j, f in enumerate(exp_series_exact(a, d)):
            out[:, i, j] = round_fraction_to_limbs(f, k)
    return out


def scalar_coeffs(rng, k: int, N: int, d: int) -> np.ndarray:
    """Degree-0 coefficient series: random k-limb scalars, higher coefficients 0."""
    c = np.zeros((k, N + 1, d + 1))
    c[:, :, 0] = random_md(rng, k, (N + 1,))
    return c


@dataclass
class SystemCase:
    """A system of polynomials sharing exp-series inputs (config 4 shape)."""
    n: int
    d: int
    k: int
    avals: list
    inputs: np.ndarray = field(repr=False)
    polys: list = field(repr=False)  # list of (supports, coeff (k, N+1, d+1))


def config4(d: int, k: int, seed: int = 0, npoly: int = 64, n: int = 64, N: int = 512,
            lo: int = 4, hi: int = 16) -> SystemCase:
    rng = np.random.default_rng(seed)
    avals = [float(a) for a in rng.uniform(-1.0, 1.0, size=n)]
    inputs = exp_inputs(avals, d, k)
    polys = []
    for _ in range(npoly):
        supp = random_supports(rng, n, N, lo, hi)
        polys.append((supp, scalar_coeffs(rng, k, N, d)))
    return SystemCase(n, d, k, avals, inputs, polys)


def binomial(n: int, r: int) -> int:
    return math.comb(n, r)
