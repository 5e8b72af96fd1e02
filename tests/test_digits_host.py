"""The library's exact digit dot product (csrc/digits.cuh, compiled for the
host) against the oracle: every convolution / correlation coefficient and every
multiple double sum must agree to far better than the per-k tolerance.

This checks the arithmetic of the convolution and addition kernels one
coefficient at a time on the CPU; the GPU tests check the kernels themselves.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_10881_gb300 import synth
from paper_2101_10881_gb300.synth import KS, random_md
from tests.exact import TOL, normwise_err

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "host", "digits_host.cpp")
LIB = os.path.join(HERE, "host", "_build", "libdigits_host.so")


@pytest.fixture(scope="module")
def dh():
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    hdr = os.path.join(HERE, "..", "paper_2101_10881_gb300", "csrc", "digits.cuh")
    if (not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", LIB, SRC], check=True)
    lib = ctypes.CDLL(LIB)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.hd_conv.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, ctypes.c_int, ctypes.c_int]
    lib.hd_sum.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
    lib.hd_conv_via_digits.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, ctypes.c_int, ctypes.c_int]
    lib.hd_sum_to_digits.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                                     ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def host_conv(dh, x, y, corr=False, bits=24):
    x = np.ascontiguousarray(x)
    y = np.ascontiguousarray(y)
    z = np.empty_like(x)
    assert dh.hd_conv(x.shape[0], x.shape[1] - 1, _p(x), _p(y), _p(z), int(corr), bits) == 0
    return z


def host_conv_via_digits(dh, x, y, corr=False, bits=28):
    x = np.ascontiguousarray(x)
    y = np.ascontiguousarray(y)
    z = np.empty_like(x)
    assert dh.hd_conv_via_digits(x.shape[0], x.shape[1] - 1, _p(x), _p(y), _p(z), int(corr), bits) == 0
    return z


def normalised(limbs):
    for a, b in zip(limbs[:-1], limbs[1:]):
        if a == 0.0:
            if b != 0.0:
                return False
        elif abs(b) > np.spacing(abs(a)) / 2:
            return False
    return True


@pytest.mark.parametrize("bits", [24, 28])
@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("d", [0, 1, 8, 40])
def test_conv_matches_oracle(dh, k, d, bits):
    rng = np.random.default_rng(10 * k + d)
    x = random_md(rng, k, (d + 1,))
    y = random_md(rng, k, (d + 1,))
    for corr in (False, True):
        z = host_conv(dh, x, y, corr, bits)
        r = O.corr(x, y) if corr else O.conv(x, y)
        assert normwise_err(z, r) <= TOL[k] * 1e-3
        for j in range(d + 1):
            assert normalised(z[:, j])


@pytest.mark.parametrize("bits", [24, 28])
@pytest.mark.parametrize("k", [1, 2, 4, 8, 10])
def test_conv_wide_dynamic_range(dh, k, bits):
    """Coefficients spanning hundreds of binary orders and exact zeros."""
    rng = np.random.default_rng(77 + k)
    d = 30
    x = random_md(rng, k, (d + 1,)) * np.ldexp(1.0, rng.integers(-300, 300, size=d + 1))
    y = random_md(rng, k, (d + 1,)) * np.ldexp(1.0, rng.integers(-300, 300, size=d + 1))
    x[:, rng.integers(0, d + 1, size=5)] = 0.0
    y[:, rng.integers(0, d + 1, size=5)] = 0.0
    z = host_conv(dh, x, y, bits=bits)
    r = O.conv(x, y)
    assert normwise_err(z, r) <= TOL[k] * 1e-3


@pytest.mark.parametrize("k", [2, 10])
def test_conv_exp_series(dh, k):
    d = 152
    z1 = synth.exp_inputs([0.75], d, k)[:, 0]
    z2 = synth.exp_inputs([-0.5], d, k)[:, 0]
    z = host_conv(dh, z1, z2)
    r = O.conv(z1, z2)
    assert normwise_err(z, r) <= TOL[k] * 1e-3


def test_conv_cancellation_exact_zero(dh):
    """(1 - t) * (1 + t + t^2 + ...) = 1 exactly: cancelled coefficients are 0."""
    k, d = 4, 20
    a = np.zeros((k, d + 1))
    a[0, 0], a[0, 1] = 1.0, -1.0
    g = np.zeros((k, d + 1))
    g[0, :] = 1.0
    z = host_conv(dh, a, g)
    assert z[0, 0] == 1.0 and np.all(z[:, 1:] == 0.0) and np.all(z[1:, 0] == 0.0)


@pytest.mark.parametrize("k", KS)
def test_sum_matches_oracle(dh, k):
    rng = np.random.default_rng(5 + k)
    for count in (1, 2, 33, 500):
        v = random_md(rng, k, (count,)) * np.ldexp(1.0, rng.integers(-40, 40, size=count))
        out = np.empty(k)
        assert dh.hd_sum(k, count, _p(np.ascontiguousarray(v)), _p(out)) == 0
        ref = O.round_sum(v.T.ravel(), k)
        assert normwise_err(out[:, None], ref[:, None]) <= TOL[k] * 1e-3
        assert normalised(out)


@pytest.mark.parametrize("bits", [24, 28])
@pytest.mark.parametrize("k", [1, 2, 10])
def test_sum_to_digits_exact(dh, k, bits):
    """Exact digit sums (words E[0..L] on grid gs) rewritten as L balanced digits
    on a grid of their own: checked in Python integers against the exact value.
    The top digit is nonzero, every digit lies in [-2^(B-1), 2^(B-1)), and the
    digits dropped below the last kept one weigh at most half its unit (plus
    one part in 2^B of it)."""
    L = dh.hd_digits_bits(k, bits)
    B = bits
    rng = np.random.default_rng(900 + 10 * k + bits)
    cases = []
    for _ in range(300):
        E = [int(v) for v in rng.integers(-(1 << 62), 1 << 62, size=L + 1)]
        cases.append(E)
    for _ in range(100):  # small words, cancellation, leading zeros
        E = [int(v) for v in rng.integers(-(1 << 20), 1 << 20, size=L + 1)]
        E[: int(rng.integers(0, L + 1))] = [0] * int(rng.integers(0, L + 1))
        cases.append(E[: L + 1] + [0] * (L + 1 - len(E[: L + 1])))
    cases.append([0] * (L + 1))
    cases.append([0] * L + [1])
    cases.append([-1] + [0] * L)
    for E in cases:
        gs = int(rng.integers(-50, 50))
        out = (ctypes.c_int32 * L)()
        grid = ctypes.c_int32()
        arr = (ctypes.c_int64 * (L + 1))(*E)
        assert dh.hd_sum_to_digits(k, bits, arr, gs, out, ctypes.byref(grid)) == 0
        # exact values scaled by 2^(B (2 L + 4 - gs)) so that everything is an integer
        sc = B * (2 * L + 4)
        V = sum(e << (sc - B * (1 + a)) for a, e in enumerate(E))  # weight 2^(B (gs - 1 - a))
        if V == 0:
            assert grid.value == -(1 << 28) and all(o == 0 for o in out)
            continue
        g = grid.value
        assert all(-(1 << (B - 1)) <= o < (1 << (B - 1)) for o in out)
        assert out[0] != 0
        # digit p weighs 2^(B (g - 1 - p)); in the scaled units: 2^(sc + B (g - gs - 1 - p))
        W = 0
        for p in range(L):
            e = sc + B * (g - gs - 1 - p)
            W += out[p] << e if e >= 0 else 0
            assert e >= 0
        unit = 1 << (sc + B * (g - gs - L))
        assert 2 * abs(V - W) <= unit + (unit >> (B - 1))


@pytest.mark.parametrize("bits", [24, 28])
@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("d", [0, 8, 40])
def test_conv_via_digits_matches_oracle(dh, k, d, bits):
    """A product kept in digit form (the workspace form of intermediate series)
    and rounded to k limbs at the end agrees with the oracle's product."""
    rng = np.random.default_rng(300 + 10 * k + d)
    x = random_md(rng, k, (d + 1,)) * np.ldexp(1.0, rng.integers(-60, 60, size=d + 1))
    y = random_md(rng, k, (d + 1,))
    for corr in (False, True):
        z = host_conv_via_digits(dh, x, y, corr, bits)
        r = O.corr(x, y) if corr else O.conv(x, y)
        assert normwise_err(z, r) <= TOL[k] * 1e-3
        for j in range(d + 1):
            assert normalised(z[:, j])
