"""Thin Python binding of libpes (include/pes.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; PyTorch is
used for device memory and streams.  The library is loaded on first use and a
missing library raises immediately: there is no CPU path.

Tensors are float64, contiguous, on the current CUDA device, in the library's
limb-major layout: coefficient series (k, N+1, d+1) with index 0 the constant
term, input series (k, n, d+1), value (k, d+1), gradient (k, n, d+1).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpes.so")

PES_OK = 0
STATUS = {0: "PES_OK", 1: "PES_EINVAL", 2: "PES_EUNSUPPORTED_K", 3: "PES_ENOMEM", 4: "PES_ECUDA",
          5: "PES_ETIMEOUT", 6: "PES_EINTERNAL", 7: "PES_EUNSUPPORTED_SIZE"}
ARITH = {"auto": -1, "fp64": 0, "int": 1}

# every symbol that include/pes.h declares
EXPORTS = ("pes_default_options", "pes_plan", "pes_plan_ex", "pes_plan_powers", "pes_plan_complex", "pes_plan_destroy",
           "pes_eval_grad", "pes_plan_system", "pes_eval_system", "pes_jobc_add_terms_system", "pes_jobc_program",
           "pes_vjp", "pes_jobc_stats_powers", "pes_jobc_jobs_powers", "pes_jobc_add_terms_powers",
           "pes_workspace_io", "pes_last_timing", "pes_batch_last_timing", "pes_check", "pes_get_plan_info", "pes_plan_batch",
           "pes_plan_batch_powers", "pes_batch_destroy",
           "pes_batch_offsets", "pes_eval_grad_batch", "pes_batch_check", "pes_get_batch_info",
           "pes_md_binary", "pes_md_costs", "pes_fp64_peak", "pes_int_peak", "pes_jobc_stats", "pes_jobc_jobs",
           "pes_jobc_add_levels", "pes_jobc_add_terms", "pes_selftest_timeout", "pes_eval_grad_static", "pes_status_string",
           "pes_last_error", "pes_shard_range", "pes_partial_grids", "pes_partial_sums", "pes_round_sums",
           "pes_round_sums_host")


class PesError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str = ""):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} {msg}".strip())


class Options(ctypes.Structure):
    _fields_ = [("arith", ctypes.c_int32), ("threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("with_vjp", ctypes.c_int32), ("timeout_ms", ctypes.c_int64), ("profile", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("staging", ctypes.c_int32), ("split", ctypes.c_int32),
                ("tile", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("conv_jobs", ctypes.c_int64), ("layers", ctypes.c_int64), ("add_terms", ctypes.c_int64),
                ("add_jobs", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
                ("vjp_conv_jobs", ctypes.c_int64), ("vjp_corr_jobs", ctypes.c_int64),
                ("digits", ctypes.c_int32), ("grid", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int32), ("arith", ctypes.c_int32), ("staging", ctypes.c_int32),
                ("split", ctypes.c_int32), ("complex_series", ctypes.c_int32), ("system_P", ctypes.c_int32),
                ("tile", ctypes.c_int32)]

    def as_dict(self):
        d = {name: int(getattr(self, name)) for name, _ in self._fields_ if name != "pad"}
        d["arith_name"] = {0: "fp64", 1: "int"}.get(d["arith"], str(d["arith"]))
        return d


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    from . import build as _b
    return _b.build(force=force)


def lib():
    """The loaded libpes (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libpes.so is not built ({LIB_PATH}); run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            i32, i64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
            ip32 = ctypes.POINTER(ctypes.c_int32)
            ip64 = ctypes.POINTER(ctypes.c_int64)
            dp = ctypes.POINTER(ctypes.c_double)
            sig = {
                "pes_default_options": (None, [ctypes.POINTER(Options)]),
                "pes_plan_ex": (i32, [ip32, ip32, i32, i32, i32, i32, ctypes.POINTER(Options), ctypes.POINTER(vp)]),
                "pes_plan_powers": (i32, [ip32, ip32, ip32, i32, i32, i32, i32, ctypes.POINTER(Options),
                                          ctypes.POINTER(vp)]),
                "pes_plan_complex": (i32, [ip32, ip32, ip32, i32, i32, i32, i32, ctypes.POINTER(Options),
                                           ctypes.POINTER(vp)]),
                "pes_plan_system": (i32, [i32, ip32, ip32, ip32, ip32, i32, i32, i32, ctypes.POINTER(Options),
                                          ctypes.POINTER(vp)]),
                "pes_eval_system": (i32, [vp, vp, vp, vp, vp, i32, vp]),
                "pes_plan_destroy": (None, [vp]),
                "pes_eval_grad": (i32, [vp, vp, vp, vp, vp, vp]),
                "pes_vjp": (i32, [vp, vp, vp, vp, vp, vp, i32, vp]),
                "pes_workspace_io": (i32, [vp, vp, i32, vp]),
                "pes_check": (i32, [vp, vp]),
                "pes_last_timing": (i32, [vp, dp, ip32]),
                "pes_batch_last_timing": (i32, [vp, dp, ip32]),
                "pes_get_plan_info": (i32, [vp, ctypes.POINTER(PlanInfo)]),
                "pes_plan_batch": (i32, [i32, ip32, ip32, ip32, ip32, ip32, i32, ctypes.POINTER(Options),
                                         ctypes.POINTER(vp)]),
                "pes_plan_batch_powers": (i32, [i32, ip32, ip32, ip32, ip32, ip32, ip32, i32,
                                                ctypes.POINTER(Options), ctypes.POINTER(vp)]),
                "pes_batch_destroy": (None, [vp]),
                "pes_batch_offsets": (i32, [vp, ip64, ip64, ip64, ip64]),
                "pes_eval_grad_batch": (i32, [vp, vp, vp, vp, vp, vp]),
                "pes_batch_check": (i32, [vp, vp]),
                "pes_get_batch_info": (i32, [vp, ctypes.POINTER(PlanInfo)]),
                "pes_md_binary": (i32, [i32, i32, vp, vp, vp, i64, vp]),
                "pes_md_costs": (i32, [i32, dp, dp]),
                "pes_fp64_peak": (i32, [i32, dp]),
                "pes_int_peak": (i32, [i32, dp]),
                "pes_jobc_stats": (i32, [ip32, ip32, i32, i32, i32, ip64, ip32, i32]),
                "pes_jobc_jobs": (i32, [ip32, ip32, i32, i32, i32, ip32, i64]),
                "pes_jobc_stats_powers": (i32, [ip32, ip32, ip32, i32, i32, i32, ip64, ip32, i32]),
                "pes_jobc_jobs_powers": (i32, [ip32, ip32, ip32, i32, i32, i32, ip32, i64]),
                "pes_jobc_add_terms_powers": (i32, [ip32, ip32, ip32, i32, i32, ip32, ip32, ip32, i64]),
                "pes_jobc_add_terms_system": (i32, [i32, ip32, ip32, ip32, ip32, i32, ip32, ip32, ip32, ip32,
                                                    i64]),
                "pes_jobc_program": (i32, [ip32, ip32, ip32, i32, i32, i32, i32, ip32, i32, ip64, ip32, ip32, ip32,
                                           ip32]),
                "pes_jobc_add_levels": (i32, [ip32, ip32, i32, i32, ip64, i32, ip32]),
                "pes_jobc_add_terms": (i32, [ip32, ip32, i32, i32, ip32, ip32, i64]),
                "pes_selftest_timeout": (i32, [i64, ip32]),
                "pes_eval_grad_static": (i32, [ip32, ip32, i32, i32, i32, i32, vp, vp, vp, vp, vp, ip32]),
                "pes_shard_range": (i32, [ip32, i32, i32, i32, ip32, ip32]),
                "pes_partial_grids": (i32, [vp, vp, vp, vp, vp]),
                "pes_partial_sums": (i32, [vp, vp, vp, vp]),
                "pes_round_sums": (i32, [vp, vp, vp, vp, vp, vp]),
                "pes_round_sums_host": (i32, [i32, i32, i32, i32, ip32, ip64, dp, dp]),
                "pes_status_string": (ctypes.c_char_p, [i32]),
                "pes_last_error": (ctypes.c_char_p, []),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc, where):
    if rc != PES_OK:
        msg = lib().pes_last_error().decode(errors="replace")
        raise PesError(rc, where, msg)


def csr(supports):
    ptr = np.zeros(len(supports) + 1, dtype=np.int32)
    idx = []
    for m, s in enumerate(supports):
        idx.extend(int(v) for v in s)
        ptr[m + 1] = len(idx)
    return ptr, np.asarray(idx if idx else [0], dtype=np.int32)


def _ip32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _iptr(t, shape, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_cuda or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


def shard_range(supports, world, rank):
    """Monomials [begin, end) that rank `rank` of `world` takes (pes_shard_range)."""
    ptr, _ = csr(supports)
    b, e = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().pes_shard_range(_ip32(ptr), len(supports), int(world), int(rank), ctypes.byref(b), ctypes.byref(e)),
           "pes_shard_range")
    return b.value, e.value


def round_sums_host(k, n, d, grids, acc, arith="int"):
    """pes_round_sums_host on numpy arrays: grids int32 (n+1, d+1), acc int64
    (n+1, d+1, L) -> value (k, d+1), grad (k, n, d+1)."""
    g = np.ascontiguousarray(grids, dtype=np.int32)
    a = np.ascontiguousarray(acc, dtype=np.int64)
    value = np.empty((k, d + 1))
    grad = np.empty((k, n, d + 1))
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib().pes_round_sums_host(int(k), ARITH[arith] if isinstance(arith, str) else int(arith), int(n), int(d),
                                     _ip32(g), a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                     value.ctypes.data_as(dp), grad.ctypes.data_as(dp)), "pes_round_sums_host")
    return value, grad


def make_options(arith="auto", threads=0, ctas_per_sm=0, with_vjp=True, timeout_ms=60000, profile=False,
                 autotune=False, staging=0, split=0, tile=0):
    o = Options()
    lib().pes_default_options(ctypes.byref(o))
    o.arith = ARITH[arith] if isinstance(arith, str) else int(arith)
    o.threads = int(threads)
    o.ctas_per_sm = int(ctas_per_sm)
    o.with_vjp = int(bool(with_vjp))
    o.timeout_ms = int(timeout_ms)
    o.profile = int(bool(profile))
    o.autotune = int(bool(autotune))
    o.staging = int(staging)
    o.split = int(split)
    o.tile = int(tile)
    return o


def _timing(fn, h, where):
    ms = (ctypes.c_double * 4)()
    nl = ctypes.c_int32()
    _check(fn(h, ms, ctypes.byref(nl)), where)
    return {"pack_ms": ms[0], "conv_ms": ms[1], "add_ms": ms[2], "unpack_ms": ms[3], "launches": nl.value}


def exponent_array(exponents, supports):
    """Flat int32 exponents aligned with csr(supports)'s index array."""
    flat = []
    assert len(exponents) == len(supports), "one exponent list per monomial"
    for s, e in zip(supports, exponents):
        assert len(e) == len(s), "one exponent per variable of the monomial"
        flat.extend(int(v) for v in e)
    return np.ascontiguousarray(np.array(flat, dtype=np.int32))


class Plan:
    """pes_plan: job tables and workspace of one polynomial on the current device.

    exponents: None (every variable with exponent 1) or, per monomial, one
    positive exponent per variable of its support (pes_plan_powers).
    complex_series: complex coefficients and inputs (pes_plan_complex); every
    buffer then has a leading axis of 2 (real part, imaginary part)."""

    def __init__(self, supports, n, d, k, exponents=None, complex_series=False, **opts):
        self.supports = [list(s) for s in supports]
        self.n, self.d, self.k = int(n), int(d), int(k)
        self.N = len(self.supports)
        self.complex_series = bool(complex_series)
        ptr, idx = csr(self.supports)
        o = make_options(**opts)
        h = ctypes.c_void_p()
        if self.complex_series:
            ex = exponent_array(exponents, self.supports) if exponents is not None else None
            _check(lib().pes_plan_complex(_ip32(ptr), _ip32(idx), _ip32(ex) if ex is not None else None, self.N,
                                          self.n, self.d, self.k, ctypes.byref(o), ctypes.byref(h)),
                   "pes_plan_complex")
        elif exponents is None:
            _check(lib().pes_plan_ex(_ip32(ptr), _ip32(idx), self.N, self.n, self.d, self.k, ctypes.byref(o),
                                     ctypes.byref(h)), "pes_plan")
        else:
            ex = exponent_array(exponents, self.supports)
            _check(lib().pes_plan_powers(_ip32(ptr), _ip32(idx), _ip32(ex), self.N, self.n, self.d, self.k,
                                         ctypes.byref(o), ctypes.byref(h)), "pes_plan_powers")
        self._h = h
        self.generation = 0  # bumped by every call that overwrites the workspace

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.pes_plan_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def shapes(self):
        k, N, n, S = self.k, self.N, self.n, self.d + 1
        sh = {"coeff": (k, N + 1, S), "input": (k, n, S), "value": (k, S), "grad": (k, n, S)}
        if getattr(self, "complex_series", False):
            sh = {key: (2,) + v for key, v in sh.items()}
        return sh

    def eval_grad(self, coeff, inputs, value=None, grad=None, stream=None):
        import torch
        sh = self.shapes()
        if value is None:
            value = torch.empty(sh["value"], dtype=torch.float64, device=coeff.device)
        if grad is None:
            grad = torch.empty(sh["grad"], dtype=torch.float64, device=coeff.device)
        _check(lib().pes_eval_grad(self._h, _ptr(coeff, sh["coeff"], "coeff"), _ptr(inputs, sh["input"], "input"),
                                   _ptr(value, sh["value"], "value"), _ptr(grad, sh["grad"], "grad"),
                                   _stream(stream)), "pes_eval_grad")
        self.generation += 1
        return value, grad

    def vjp(self, coeff, inputs, upstream, reuse_forward=False, grad_input=None, grad_coeff=None, stream=None):
        import torch
        sh = self.shapes()
        dev = upstream.device
        if grad_input is None:
            grad_input = torch.empty(sh["input"], dtype=torch.float64, device=dev)
        if grad_coeff is None:
            grad_coeff = torch.empty(sh["coeff"], dtype=torch.float64, device=dev)
        cp = _ptr(coeff, sh["coeff"], "coeff") if coeff is not None else ctypes.c_void_p(0)
        ip = _ptr(inputs, sh["input"], "input") if inputs is not None else ctypes.c_void_p(0)
        _check(lib().pes_vjp(self._h, cp, ip, _ptr(upstream, sh["value"], "upstream"),
                             _ptr(grad_input, sh["input"], "grad_input"),
                             _ptr(grad_coeff, sh["coeff"], "grad_coeff"), int(bool(reuse_forward)),
                             _stream(stream)), "pes_vjp")
        self.generation += 1
        return grad_input, grad_coeff

    # ---- partial sums of a polynomial split over ranks (pes_partial_*) ----

    def partial_grids(self, coeff, inputs, grids=None, stream=None):
        """Convolutions of this plan, then the largest grid of every output
        coefficient's contributions: int32 (n+1, d+1), row 0 the value."""
        import torch
        sh = self.shapes()
        if grids is None:
            grids = torch.empty((self.n + 1, self.d + 1), dtype=torch.int32, device=coeff.device)
        _check(lib().pes_partial_grids(self._h, _ptr(coeff, sh["coeff"], "coeff"), _ptr(inputs, sh["input"], "input"),
                                       _iptr(grids, (self.n + 1, self.d + 1), torch.int32, "grids"),
                                       _stream(stream)), "pes_partial_grids")
        return grids

    def partial_sums(self, grids, acc=None, stream=None):
        """Exact digit sums of every output coefficient on the given grids:
        int64 (n+1, d+1, L), unrounded."""
        import torch
        L = self.info()["digits"]
        if acc is None:
            acc = torch.empty((self.n + 1, self.d + 1, L), dtype=torch.int64, device=grids.device)
        _check(lib().pes_partial_sums(self._h, _iptr(grids, (self.n + 1, self.d + 1), torch.int32, "grids"),
                                      _iptr(acc, (self.n + 1, self.d + 1, L), torch.int64, "acc"),
                                      _stream(stream)), "pes_partial_sums")
        return acc

    def round_sums(self, grids, acc, value=None, grad=None, stream=None):
        """Digit sums (summed over the ranks) rounded once to k limbs."""
        import torch
        sh = self.shapes()
        L = self.info()["digits"]
        if value is None:
            value = torch.empty(sh["value"], dtype=torch.float64, device=grids.device)
        if grad is None:
            grad = torch.empty(sh["grad"], dtype=torch.float64, device=grids.device)
        _check(lib().pes_round_sums(self._h, _iptr(grids, (self.n + 1, self.d + 1), torch.int32, "grids"),
                                    _iptr(acc, (self.n + 1, self.d + 1, L), torch.int64, "acc"),
                                    _ptr(value, sh["value"], "value"), _ptr(grad, sh["grad"], "grad"),
                                    _stream(stream)), "pes_round_sums")
        return value, grad

    def workspace_io(self, buffer, to_buffer, stream=None):
        _check(lib().pes_workspace_io(self._h, ctypes.c_void_p(buffer.data_ptr()), int(bool(to_buffer)),
                                      _stream(stream)), "pes_workspace_io")

    def check(self, stream=None):
        _check(lib().pes_check(self._h, _stream(stream)), "pes_check")

    def last_timing(self):
        """Per-phase device time of the last call (plan built with profile=True)."""
        return _timing(lib().pes_last_timing, self._h, "pes_last_timing")

    def info(self):
        pi = PlanInfo()
        _check(lib().pes_get_plan_info(self._h, ctypes.byref(pi)), "pes_get_plan_info")
        return pi.as_dict()


LAYOUTS = {"series": 0, "matrix": 1}


class System(Plan):
    """pes_plan_system: P polynomials in the same n variables, their values and
    their Jacobian matrix at the input series in one job table.

    polys: list of P polynomials, each a list of supports (variable-index
    lists); exponents: None or, per polynomial, per monomial, one positive
    exponent per variable.  The coefficient buffer is [k][N+P][d+1]: each
    polynomial's constant series, then its monomials' coefficient series.
    Differentiable through autograd.poly_eval (one upstream series per
    polynomial)."""

    def __init__(self, polys, n, d, k, exponents=None, **opts):
        self.polys = [[list(m) for m in p_] for p_ in polys]
        self.P = len(self.polys)
        self.supports = [m for p_ in self.polys for m in p_]
        self.n, self.d, self.k = int(n), int(d), int(k)
        self.N = len(self.supports)
        self.complex_series = False
        self.poly_ptr = np.zeros(self.P + 1, dtype=np.int32)
        self.poly_ptr[1:] = np.cumsum([len(p_) for p_ in self.polys])
        ptr, idx = csr(self.supports)
        ex = None
        if exponents is not None:
            ex = exponent_array([e for pe in exponents for e in pe], self.supports)
        o = make_options(**opts)
        h = ctypes.c_void_p()
        _check(lib().pes_plan_system(self.P, _ip32(self.poly_ptr), _ip32(ptr), _ip32(idx),
                                     _ip32(ex) if ex is not None and ex.size else None, self.n, self.d, self.k,
                                     ctypes.byref(o), ctypes.byref(h)), "pes_plan_system")
        self._h = h
        self.generation = 0

    def coeff_index(self, p, m=None):
        """Row of the coefficient buffer: polynomial p's constant (m None) or
        its monomial m (0-based within p)."""
        base = int(self.poly_ptr[p]) + p
        return base if m is None else base + 1 + m

    def shapes(self, layout="series"):
        k, N, n, P, S = self.k, self.N, self.n, self.P, self.d + 1
        sh = {"coeff": (k, N + P, S), "input": (k, n, S)}
        if layout == "series":
            sh.update(value=(k, P, S), jac=(k, P, n, S))
        else:
            sh.update(value=(k, S, P), jac=(k, S, P, n))
        return sh

    def eval_system(self, coeff, inputs, layout="series", value=None, jac=None, stream=None):
        import torch
        sh = self.shapes(layout)
        if value is None:
            value = torch.empty(sh["value"], dtype=torch.float64, device=coeff.device)
        if jac is None:
            jac = torch.empty(sh["jac"], dtype=torch.float64, device=coeff.device)
        _check(lib().pes_eval_system(self._h, _ptr(coeff, sh["coeff"], "coeff"), _ptr(inputs, sh["input"], "input"),
                                     _ptr(value, sh["value"], "value"), _ptr(jac, sh["jac"], "jac"),
                                     LAYOUTS[layout], _stream(stream)), "pes_eval_system")
        self.generation += 1
        return value, jac

    def eval_grad(self, coeff, inputs, value=None, grad=None, stream=None):
        return self.eval_system(coeff, inputs, "series", value, grad, stream)

    # vjp (Plan.vjp): upstream (k, P, d+1), one series per polynomial; returns
    # grad_input (k, n, d+1) and grad_coeff (k, N+P, d+1)


class Batch:
    """pes_plan_batch: many polynomials evaluated by one graph-captured launch."""

    def __init__(self, instances, k, exponents=None, **opts):
        """instances: list of (supports, n, d); exponents: None or, per
        instance, per monomial, one positive exponent per variable."""
        self.k = int(k)
        self.count = len(instances)
        n = np.array([int(t[1]) for t in instances], dtype=np.int32)
        d = np.array([int(t[2]) for t in instances], dtype=np.int32)
        N = np.array([len(t[0]) for t in instances], dtype=np.int32)
        ptrs, idxs, exs = [], [], []
        for b, (supp, _, _) in enumerate(instances):
            p, i = csr(supp)
            ptrs.append(p)
            idxs.append(i[: p[-1]])
            if exponents is not None:
                exs.append(exponent_array(exponents[b], supp))
        ptr = np.concatenate(ptrs).astype(np.int32)
        idx = np.concatenate(idxs).astype(np.int32) if sum(len(x) for x in idxs) else np.zeros(1, np.int32)
        ex = None
        if exponents is not None:
            ex = np.concatenate(exs).astype(np.int32) if sum(len(x) for x in exs) else np.ones(1, np.int32)
        o = make_options(**opts)
        h = ctypes.c_void_p()
        _check(lib().pes_plan_batch_powers(self.count, _ip32(n), _ip32(N), _ip32(d), _ip32(ptr), _ip32(idx),
                                           _ip32(ex) if ex is not None else None, self.k, ctypes.byref(o),
                                           ctypes.byref(h)), "pes_plan_batch_powers")
        self._h = h
        self.n, self.N, self.d = n, N, d
        offs = [np.zeros(self.count + 1, dtype=np.int64) for _ in range(4)]
        p64 = [o_.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)) for o_ in offs]
        _check(lib().pes_batch_offsets(self._h, *p64), "pes_batch_offsets")
        self.coeff_off, self.input_off, self.value_off, self.grad_off = offs

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.pes_batch_destroy(h)
            self._h = None

    def lengths(self):
        return {"coeff": int(self.coeff_off[-1]), "input": int(self.input_off[-1]),
                "value": int(self.value_off[-1]), "grad": int(self.grad_off[-1])}

    def eval_grad(self, coeff, inputs, value, grad, stream=None):
        ln = self.lengths()
        _check(lib().pes_eval_grad_batch(self._h, _ptr(coeff, (ln["coeff"],), "coeff"),
                                         _ptr(inputs, (ln["input"],), "input"),
                                         _ptr(value, (ln["value"],), "value"), _ptr(grad, (ln["grad"],), "grad"),
                                         _stream(stream)), "pes_eval_grad_batch")
        return value, grad

    def check(self, stream=None):
        _check(lib().pes_batch_check(self._h, _stream(stream)), "pes_batch_check")

    def last_timing(self):
        return _timing(lib().pes_batch_last_timing, self._h, "pes_batch_last_timing")

    def info(self):
        pi = PlanInfo()
        _check(lib().pes_get_batch_info(self._h, ctypes.byref(pi)), "pes_get_batch_info")
        return pi.as_dict()


def md_binary(op, x, y, out=None, stream=None):
    """Elementwise k-double add (op 'add') or mul (op 'mul') of (k, count) tensors."""
    import torch
    k, count = x.shape
    if out is None:
        out = torch.empty_like(x)
    _check(lib().pes_md_binary({"add": 0, "mul": 1}[op], k, _ptr(x, (k, count), "x"), _ptr(y, (k, count), "y"),
                               _ptr(out, (k, count), "out"), count, _stream(stream)), "pes_md_binary")
    return out


def md_costs(k):
    m, a = ctypes.c_double(), ctypes.c_double()
    _check(lib().pes_md_costs(int(k), ctypes.byref(m), ctypes.byref(a)), "pes_md_costs")
    return m.value, a.value


def fp64_peak(repeats=5):
    t = ctypes.c_double()
    _check(lib().pes_fp64_peak(int(repeats), ctypes.byref(t)), "pes_fp64_peak")
    return t.value


def int_peak(repeats=5):
    t = ctypes.c_double()
    _check(lib().pes_int_peak(int(repeats), ctypes.byref(t)), "pes_int_peak")
    return t.value


def jobc_stats(supports, n, paper_layout=False, max_layers=4096, exponents=None):
    ptr, idx = csr(supports)
    stats = np.zeros(8, dtype=np.int64)
    layers = np.zeros(max_layers, dtype=np.int32)
    sp = stats.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    if exponents is None:
        _check(lib().pes_jobc_stats(_ip32(ptr), _ip32(idx), len(supports), int(n), int(bool(paper_layout)),
                                    sp, _ip32(layers), max_layers), "pes_jobc_stats")
    else:
        ex = exponent_array(exponents, supports)
        _check(lib().pes_jobc_stats_powers(_ip32(ptr), _ip32(idx), _ip32(ex), len(supports), int(n),
                                           int(bool(paper_layout)), sp, _ip32(layers), max_layers),
               "pes_jobc_stats_powers")
    keys = ("conv_jobs", "layers", "add_terms", "paper_add_jobs", "slots", "add_levels", "vjp_conv", "vjp_corr")
    out = {k_: int(v) for k_, v in zip(keys, stats)}
    out["layer_sizes"] = [int(v) for v in layers[: out["layers"]]]
    return out


def jobc_jobs(supports, n, paper_layout=False, exponents=None):
    st = jobc_stats(supports, n, paper_layout, exponents=exponents)
    ptr, idx = csr(supports)
    jobs = np.zeros((max(st["conv_jobs"], 1), 4), dtype=np.int32)
    if exponents is None:
        _check(lib().pes_jobc_jobs(_ip32(ptr), _ip32(idx), len(supports), int(n), int(bool(paper_layout)),
                                   _ip32(jobs), st["conv_jobs"]), "pes_jobc_jobs")
    else:
        ex = exponent_array(exponents, supports)
        _check(lib().pes_jobc_jobs_powers(_ip32(ptr), _ip32(idx), _ip32(ex), len(supports), int(n),
                                          int(bool(paper_layout)), _ip32(jobs), st["conv_jobs"]),
               "pes_jobc_jobs_powers")
    return jobs[: st["conv_jobs"]]


def jobc_add_levels(supports, n, cap=256):
    ptr, idx = csr(supports)
    lv = np.zeros(cap, dtype=np.int64)
    nl = ctypes.c_int32()
    _check(lib().pes_jobc_add_levels(_ip32(ptr), _ip32(idx), len(supports), int(n),
                                     lv.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cap, ctypes.byref(nl)),
           "pes_jobc_add_levels")
    return [int(v) for v in lv[: nl.value]]


def jobc_add_terms(supports, n, exponents=None):
    """(add_ptr, add_src), and add_mult as well when exponents are given."""
    st = jobc_stats(supports, n, exponents=exponents)
    ptr, idx = csr(supports)
    add_ptr = np.zeros(int(n) + 2, dtype=np.int32)
    add_src = np.zeros(max(st["add_terms"], 1), dtype=np.int32)
    if exponents is None:
        _check(lib().pes_jobc_add_terms(_ip32(ptr), _ip32(idx), len(supports), int(n), _ip32(add_ptr),
                                        _ip32(add_src), st["add_terms"]), "pes_jobc_add_terms")
        return add_ptr, add_src[: st["add_terms"]]
    add_mult = np.zeros(max(st["add_terms"], 1), dtype=np.int32)
    ex = exponent_array(exponents, supports)
    _check(lib().pes_jobc_add_terms_powers(_ip32(ptr), _ip32(idx), _ip32(ex), len(supports), int(n),
                                           _ip32(add_ptr), _ip32(add_src), _ip32(add_mult), st["add_terms"]),
           "pes_jobc_add_terms_powers")
    return add_ptr, add_src[: st["add_terms"]], add_mult[: st["add_terms"]]


def jobc_add_terms_system(polys, n, exponents=None):
    """(const0, add_ptr, add_src, add_mult) of a system (pes_jobc_add_terms_system):
    outputs p < P the values, P + p*n + i the Jacobian entries."""
    supports = [m for p_ in polys for m in p_]
    P = len(polys)
    poly_ptr = np.zeros(P + 1, dtype=np.int32)
    poly_ptr[1:] = np.cumsum([len(p_) for p_ in polys])
    flat_ex = [e for pe in exponents for e in pe] if exponents is not None else None
    cap = jobc_stats(supports, n, exponents=flat_ex)["add_terms"] + P
    ptr, idx = csr(supports)
    ex = exponent_array(flat_ex, supports) if flat_ex is not None else None
    const0 = ctypes.c_int32()
    add_ptr = np.zeros(P + P * int(n) + 1, dtype=np.int32)
    add_src = np.zeros(cap, dtype=np.int32)
    add_mult = np.zeros(cap, dtype=np.int32)
    _check(lib().pes_jobc_add_terms_system(P, _ip32(poly_ptr), _ip32(ptr), _ip32(idx),
                                           _ip32(ex) if ex is not None and ex.size else None, int(n),
                                           ctypes.byref(const0), _ip32(add_ptr), _ip32(add_src), _ip32(add_mult),
                                           cap), "pes_jobc_add_terms_system")
    nt = int(add_ptr[-1])
    return const0.value, add_ptr, add_src[:nt], add_mult[:nt]


def jobc_program(supports, n, exponents=None, complex_series=False, with_vjp=False, polys=None):
    """The whole program of a plan as host tables (pes_jobc_program): a dict with
    jobs (rows of in1, in2, out, layer, kind; evaluation then VJP), the addition
    tables, the slot counts and the VJP slot numbers.  polys: for a system, the
    number of monomials of each polynomial (supports in that order)."""
    ptr, idx = csr(supports)
    ex = exponent_array(exponents, supports) if exponents is not None else None
    exp_p = _ip32(ex) if ex is not None and ex.size else None
    P = 0 if polys is None else len(polys)
    poly_ptr = np.zeros(P + 1, dtype=np.int32)
    if P:
        poly_ptr[1:] = np.cumsum(polys)
    counts = np.zeros(14, dtype=np.int64)
    args = (_ip32(ptr), _ip32(idx), exp_p, len(supports), int(n), int(bool(complex_series)), P,
            _ip32(poly_ptr) if P else None, int(bool(with_vjp)))
    c64 = counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    _check(lib().pes_jobc_program(*args, c64, None, None, None, None), "pes_jobc_program")
    nj = int(counts[0] + counts[4])
    jobs = np.zeros((max(nj, 1), 5), dtype=np.int32)
    add_ptr = np.zeros(int(counts[1]) + 1, dtype=np.int32)
    add_src = np.zeros(max(int(counts[2]), 1), dtype=np.int32)
    add_mult = np.zeros(max(int(counts[2]), 1), dtype=np.int32)
    _check(lib().pes_jobc_program(*args, c64, _ip32(jobs), _ip32(add_ptr), _ip32(add_src), _ip32(add_mult)),
           "pes_jobc_program")
    ne = int(counts[0])
    return {"jobs": jobs[:ne], "vjp_jobs": jobs[ne:nj], "vjp_fwd_jobs": int(counts[5]),
            "add_ptr": add_ptr, "add_src": add_src[: int(counts[2])], "add_mult": add_mult[: int(counts[2])],
            "slots": int(counts[3]), "slot_u": int(counts[6]), "slot_g0": int(counts[7]),
            "slot_r0": int(counts[8]), "input_slots": int(counts[9]), "const0": int(counts[10]),
            "slot_up0": int(counts[11]), "slot_J0": int(counts[12]), "slot_rJ0": int(counts[13])}


def selftest_timeout(timeout_ms=500):
    """Run the bounded-wait failure path; returns the device status it reported."""
    status = ctypes.c_int32(-1)
    _check(lib().pes_selftest_timeout(int(timeout_ms), ctypes.byref(status)), "pes_selftest_timeout")
    return STATUS.get(status.value, status.value)
