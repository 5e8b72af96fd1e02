"""pes_eval_grad_static: evaluation and differentiation for callers that cannot
allocate device memory (code inside another framework's memory pool, plug-ins
whose host forbids device allocations, paths that must keep the device
footprint fixed).  The entry point keeps its tables and workspace in a fixed
static device array of the library instead of calling cudaMalloc.  It must give
the same bits as the allocating path (pes_plan + pes_eval_grad), call after
call, since every call reuses and rewrites the same array, and it must not
change the device's free memory.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes when run alone.
"""
import ctypes

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


def outputs(torch, prob):
    v = torch.empty((prob.k, prob.d + 1), dtype=torch.float64, device="cuda")
    g = torch.empty((prob.k, prob.n, prob.d + 1), dtype=torch.float64, device="cuda")
    return v, g


def static_rc(torch, prob, coeff, inputs, v, g, status=None):
    """Call the allocation-free entry point through the C-ABI; its status code."""
    ptr, idx = pes.csr(prob.supports)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return pes.lib().pes_eval_grad_static(
        ptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
        prob.N, prob.n, prob.d, prob.k, ctypes.c_void_p(coeff.data_ptr()), ctypes.c_void_p(inputs.data_ptr()),
        ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(g.data_ptr()), stream,
        ctypes.byref(status) if status is not None else None)


def static_call(torch, prob, coeff, inputs, v, g):
    status = ctypes.c_int32(-1)
    rc = static_rc(torch, prob, coeff, inputs, v, g, status)
    assert rc == 0, pes.lib().pes_last_error()
    assert status.value == 0
    return v.cpu().numpy(), g.cpu().numpy()


def problems():
    rng = np.random.default_rng(2024)
    small = synth.Problem("k10", 9, 40, 10, synth.random_supports(rng, 9, 14, 1, 6),
                          random_md(rng, 10, (15, 41)), random_md(rng, 10, (9, 41)))
    return [synth.config0(seed=3), small]


@pytest.mark.parametrize("case", [0, 1])
def test_static_entry_matches_allocating_path(torch, case):
    """Two calls in a row give the allocating path's bits (the same exact sums
    rounded once) and agree with the oracle within the per-k tolerance; the
    second call leaves the device's free memory unchanged."""
    prob = problems()[case]
    C = torch.from_numpy(prob.coeff).cuda()
    Z = torch.from_numpy(prob.inputs).cuda()
    plan = pes.Plan(prob.supports, prob.n, prob.d, prob.k)
    rv, rg = plan.eval_grad(C, Z)
    plan.check()
    rv, rg = rv.cpu().numpy(), rg.cpu().numpy()
    v, g = outputs(torch, prob)
    first = static_call(torch, prob, C, Z, v, g)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    second = static_call(torch, prob, C, Z, v, g)  # the array keeps the last call's contents
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    ov, og = O.eval_grad(prob.supports, prob.n, prob.coeff, prob.inputs)
    for sv, sg in (first, second):
        assert np.array_equal(sv, rv) and np.array_equal(sg, rg)
        assert normwise_err(sv, ov) <= TOL[prob.k]
        assert normwise_err(sg, og) <= TOL[prob.k]


def test_static_entry_rejects_oversized_problem(torch):
    prob = synth.config1()  # the deca double workload needs ~460 MB of workspace
    C = torch.from_numpy(prob.coeff).cuda()
    Z = torch.from_numpy(prob.inputs).cuda()
    v, g = outputs(torch, prob)
    assert static_rc(torch, prob, C, Z, v, g) == 7  # PES_EUNSUPPORTED_SIZE
    assert b"scratch" in pes.lib().pes_last_error()


@pytest.mark.parametrize("k,d", [(2, 1024), (10, 472)])
def test_static_entry_rejects_large_degrees(torch, k, d):
    """Above d = 1023, and above the degree whose whole series fit one CTA's
    shared memory (471 at k = 10), the call is refused with
    PES_EUNSUPPORTED_SIZE before anything is enqueued."""
    rng = np.random.default_rng(d)
    prob = synth.Problem("big", 2, d, k, [[0, 1]], random_md(rng, k, (2, d + 1)), random_md(rng, k, (2, d + 1)))
    C = torch.from_numpy(prob.coeff).cuda()
    Z = torch.from_numpy(prob.inputs).cuda()
    v, g = outputs(torch, prob)
    assert static_rc(torch, prob, C, Z, v, g) == 7
    assert pes.lib().pes_last_error()
