"""Python handle on the oracle (pes_oracle.c): test infrastructure only.

The oracle is the plain CPU restatement of what the library computes (Verschelde
2021, Eq. (eqconvform) for the truncated series product and Eq. (eqpolynomial)
for the polynomial and its gradient).  Only tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline and reference legs use it; the product path never does.

Arrays follow the library's limb-major layout: a series array is float64 of
shape (k, n_series, d+1); a single series is (k, d+1); a multiple double scalar
is (k,).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pes_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# -ffp-contract=off: Dekker's TwoProduct and Knuth's TwoSum must not be fused
# into multiply-adds by the compiler.
CFLAGS = ["-O2", "-fPIC", "-shared", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fopenmp"]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to this file (gcc, a second or two)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)
            c_int = ctypes.c_int
            for name, args in {
                "orc_md_add": [c_int, dp, dp, dp],
                "orc_md_mul": [c_int, dp, dp, dp],
                "orc_round_sum": [c_int, c_int, dp, dp],
                "orc_conv": [c_int, c_int, dp, dp, dp],
                "orc_corr": [c_int, c_int, dp, dp, dp],
                "orc_eval_grad": [c_int, c_int, c_int, c_int, ip, ip, dp, dp, dp, dp, c_int],
                "orc_vjp": [c_int, c_int, c_int, c_int, ip, ip, dp, dp, dp, dp, dp, c_int],
                "orc_eval_grad_pow": [c_int, c_int, c_int, c_int, ip, ip, ip, dp, dp, dp, dp, c_int],
                "orc_vjp_pow": [c_int, c_int, c_int, c_int, ip, ip, ip, dp, dp, dp, dp, dp, c_int],
                "orc_eval_grad_complex": [c_int, c_int, c_int, c_int, ip, ip, ip, dp, dp, dp, dp],
                "orc_vjp_complex": [c_int, c_int, c_int, c_int, ip, ip, ip, dp, dp, dp, dp, dp],
                "orc_threads": [c_int],
                "orc_conv_many": [c_int, c_int, c_int, dp, dp, dp, c_int],
            }.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = c_int
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def md_add(x, y):
    x, y = _f64(x), _f64(y)
    k = x.shape[0]
    out = np.empty(k)
    _check(_load().orc_md_add(k, _dp(x), _dp(y), _dp(out)), "md_add")
    return out


def md_mul(x, y):
    x, y = _f64(x), _f64(y)
    k = x.shape[0]
    out = np.empty(k)
    _check(_load().orc_md_mul(k, _dp(x), _dp(y), _dp(out)), "md_mul")
    return out


def round_sum(values, k):
    """round_k of the exact sum of a list of doubles."""
    v = _f64(values).ravel()
    out = np.empty(k)
    _check(_load().orc_round_sum(k, v.size, _dp(v), _dp(out)), "round_sum")
    return out


def conv(x, y):
    """Truncated product of two series, (k, d+1) each."""
    x, y = _f64(x), _f64(y)
    k, s = x.shape
    z = np.empty_like(x)
    _check(_load().orc_conv(k, s - 1, _dp(x), _dp(y), _dp(z)), "conv")
    return z


def conv_many(x, y, nthreads: int = 0):
    """Independent truncated products of (k, count, d+1) arrays, pairwise."""
    x, y = _f64(x), _f64(y)
    k, count, s = x.shape
    z = np.empty_like(x)
    _check(_load().orc_conv_many(k, s - 1, count, _dp(x), _dp(y), _dp(z), nthreads), "conv_many")
    return z


def corr(u, s):
    """Truncated correlation r_j = sum_{l>=j} u_l s_{l-j}, (k, d+1) each."""
    u, s = _f64(u), _f64(s)
    k, n = u.shape
    r = np.empty_like(u)
    _check(_load().orc_corr(k, n - 1, _dp(u), _dp(s), _dp(r)), "corr")
    return r


def _supports(supports):
    ptr = np.zeros(len(supports) + 1, dtype=np.int32)
    idx = []
    for m, s in enumerate(supports):
        idx.extend(int(v) for v in s)
        ptr[m + 1] = len(idx)
    return ptr, np.asarray(idx, dtype=np.int32)


def _exponents(exponents, supports):
    """Flat int32 exponents aligned with the supports (None: all 1)."""
    if exponents is None:
        return None
    assert len(exponents) == len(supports)
    flat = []
    for s, e in zip(supports, exponents):
        assert len(e) == len(s)
        flat.extend(int(v) for v in e)
    return np.ascontiguousarray(np.array(flat, dtype=np.int32))


def eval_grad(supports, n, coeff, inputs, nthreads: int = 0, grad: bool = True, exponents=None):
    """Value (k, d+1) and gradient (k, n, d+1) of the polynomial at the series.

    supports: list of increasing 0-based variable index lists, one per monomial.
    exponents: None (every exponent 1) or one list of positive exponents per
    monomial, aligned with its support.
    coeff: (k, N+1, d+1) with index 0 the constant term; inputs: (k, n, d+1).
    """
    coeff, inputs = _f64(coeff), _f64(inputs)
    k, n1, s = coeff.shape
    N = len(supports)
    assert n1 == N + 1 and inputs.shape == (k, n, s)
    ptr, idx = _supports(supports)
    ex = _exponents(exponents, supports)
    value = np.empty((k, s))
    g = np.empty((k, n, s)) if grad else None
    gp = _dp(g) if grad else ctypes.POINTER(ctypes.c_double)()
    if ex is None:
        _check(_load().orc_eval_grad(k, s - 1, N, n, _ip(ptr), _ip(idx), _dp(coeff), _dp(inputs),
                                     _dp(value), gp, nthreads), "eval_grad")
    else:
        _check(_load().orc_eval_grad_pow(k, s - 1, N, n, _ip(ptr), _ip(idx), _ip(ex), _dp(coeff),
                                         _dp(inputs), _dp(value), gp, nthreads), "eval_grad_pow")
    return (value, g) if grad else value


def eval_grad_complex(supports, n, coeff, inputs, exponents=None, grad: bool = True):
    """Complex coefficients and inputs: coeff (2, k, N+1, d+1), inputs
    (2, k, n, d+1), index 0 of the first axis the real part.  Returns value
    (2, k, d+1) and gradient (2, k, n, d+1)."""
    coeff, inputs = _f64(coeff), _f64(inputs)
    two, k, n1, s = coeff.shape
    N = len(supports)
    assert two == 2 and n1 == N + 1 and inputs.shape == (2, k, n, s)
    ptr, idx = _supports(supports)
    ex = _exponents(exponents, supports)
    exp_p = _ip(ex) if ex is not None else ctypes.POINTER(ctypes.c_int32)()
    value = np.empty((2, k, s))
    g = np.empty((2, k, n, s)) if grad else None
    gp = _dp(g) if grad else ctypes.POINTER(ctypes.c_double)()
    _check(_load().orc_eval_grad_complex(k, s - 1, N, n, _ip(ptr), _ip(idx), exp_p, _dp(coeff), _dp(inputs),
                                         _dp(value), gp), "eval_grad_complex")
    return (value, g) if grad else value


def vjp_complex(supports, n, coeff, inputs, upstream, exponents=None):
    """(grad_input (2, k, n, d+1), grad_coeff (2, k, N+1, d+1)) of the real loss
    L = sum_j (Re u_j Re v_j + Im u_j Im v_j), upstream u (2, k, d+1): the
    derivatives with respect to the real parts (index 0) and the imaginary
    parts (index 1) of every input and coefficient series."""
    coeff, inputs, upstream = _f64(coeff), _f64(inputs), _f64(upstream)
    two, k, n1, s = coeff.shape
    N = len(supports)
    assert two == 2 and n1 == N + 1 and inputs.shape == (2, k, n, s) and upstream.shape == (2, k, s)
    ptr, idx = _supports(supports)
    ex = _exponents(exponents, supports)
    exp_p = _ip(ex) if ex is not None else ctypes.POINTER(ctypes.c_int32)()
    gi = np.empty((2, k, n, s))
    gc = np.empty((2, k, N + 1, s))
    _check(_load().orc_vjp_complex(k, s - 1, N, n, _ip(ptr), _ip(idx), exp_p, _dp(coeff), _dp(inputs),
                                   _dp(upstream), _dp(gi), _dp(gc)), "vjp_complex")
    return gi, gc


def vjp(supports, n, coeff, inputs, upstream, nthreads: int = 0, exponents=None):
    """(grad_input (k, n, d+1), grad_coeff (k, N+1, d+1)) of <upstream, value>."""
    coeff, inputs, upstream = _f64(coeff), _f64(inputs), _f64(upstream)
    k, n1, s = coeff.shape
    N = len(supports)
    ptr, idx = _supports(supports)
    ex = _exponents(exponents, supports)
    gi = np.empty((k, n, s))
    gc = np.empty((k, N + 1, s))
    if ex is None:
        _check(_load().orc_vjp(k, s - 1, N, n, _ip(ptr), _ip(idx), _dp(coeff), _dp(inputs),
                               _dp(upstream), _dp(gi), _dp(gc), nthreads), "vjp")
    else:
        _check(_load().orc_vjp_pow(k, s - 1, N, n, _ip(ptr), _ip(idx), _ip(ex), _dp(coeff), _dp(inputs),
                                   _dp(upstream), _dp(gi), _dp(gc), nthreads), "vjp_pow")
    return gi, gc


def threads(nthreads: int = 0) -> int:
    return int(_load().orc_threads(nthreads))
