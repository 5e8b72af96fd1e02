"""pes_eval_grad_static: evaluation and differentiation for callers that cannot
allocate device memory (code inside another framework's memory pool, plug-ins
whose host forbids device allocations).  The entry point keeps its tables and
workspace in a fixed static device array of the library instead of calling
cudaMalloc.  It must give the same values as the allocating path
(pes_plan + pes_eval_grad), call after call, since every call reuses and
rewrites the same array.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes when run alone.
"""
import ctypes

import numpy as np
import pytest

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


def static_call(torch, prob, coeff, inputs):
    """Call the allocation-free entry point through the C-ABI."""
    ptr, idx = pes.csr(prob.supports)
    v = torch.empty((prob.k, prob.d + 1), dtype=torch.float64, device="cuda")
    g = torch.empty((prob.k, prob.n, prob.d + 1), dtype=torch.float64, device="cuda")
    status = ctypes.c_int32(-1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = pes.lib().pes_eval_grad_static(
        ptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
        prob.N, prob.n, prob.d, prob.k, ctypes.c_void_p(coeff.data_ptr()), ctypes.c_void_p(inputs.data_ptr()),
        ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(g.data_ptr()), stream, ctypes.byref(status))
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
    prob = problems()[case]
    C = torch.from_numpy(prob.coeff).cuda()
    Z = torch.from_numpy(prob.inputs).cuda()
    plan = pes.Plan(prob.supports, prob.n, prob.d, prob.k)
    rv, rg = plan.eval_grad(C, Z)
    plan.check()
    rv, rg = rv.cpu().numpy(), rg.cpu().numpy()
    first = static_call(torch, prob, C, Z)
    second = static_call(torch, prob, C, Z)  # the array keeps the last call's contents
    for v, g in (first, second):
        assert normwise_err(v, rv) <= TOL[prob.k]
        assert normwise_err(g, rg) <= TOL[prob.k]
    assert np.array_equal(first[0], second[0]) and np.array_equal(first[1], second[1])


def test_static_entry_rejects_oversized_problem(torch):
    prob = synth.config1()  # the deca double workload needs ~320 MB of workspace
    C = torch.from_numpy(prob.coeff).cuda()
    Z = torch.from_numpy(prob.inputs).cuda()
    ptr, idx = pes.csr(prob.supports)
    v = torch.empty((prob.k, prob.d + 1), dtype=torch.float64, device="cuda")
    g = torch.empty((prob.k, prob.n, prob.d + 1), dtype=torch.float64, device="cuda")
    rc = pes.lib().pes_eval_grad_static(
        ptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
        prob.N, prob.n, prob.d, prob.k, ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(Z.data_ptr()),
        ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(0), None)
    assert rc == 7  # PES_EUNSUPPORTED_SIZE
    assert b"scratch" in pes.lib().pes_last_error()
