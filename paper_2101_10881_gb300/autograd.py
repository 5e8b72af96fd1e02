"""torch.autograd for polynomial evaluation at power series in k-double precision.

Tensors here hold k-double series in the library's limb-major layout: a tensor
of shape (k, ..., d+1) represents, for every series and coefficient, the single
number sum_l t[l, ..., j].  Gradients follow the same convention: the gradient
returned for `coeff` is the k-double series dL/da (limb-major, shape of
`coeff`), and the upstream gradient of `value` is read as the k-double series
u = dL/dv.  For L = sum_j v_j^2, for example, call `value.backward(2 * value)`:
doubling every limb doubles the k-double exactly.

Forward: pes_eval_grad (the reverse mode of Sec. 3, layered jobs of Sec. 5).
Backward: pes_vjp, a hand-written kernel path computing the vector-Jacobian
product by truncated correlations (transposed convolutions):
    dL/da_0[j] = u_j,  dL/da_m[j] = sum_{l>=j} u_l M_m[l-j],  dL/dz_i[j] = sum_{l>=j} u_l g_i[l-j],
with M_m the product of the variables of monomial m and g_i = dp/dx_i; exact
because every variable has exponent 1, so v is affine in each series.

PyTorch adds the gradients of a tensor that feeds several calls limb by limb,
which is double-precision addition of the limbs, not k-double addition; for
several polynomials in the same inputs use one pes.System, whose single VJP sums
the input gradients over the polynomials exactly and rounds once.

Forward products are reused when possible: if no other call ran on the plan
since the forward, the plan's workspace still holds them; otherwise, if the
workspace fit `memory_budget` bytes at forward time, a snapshot taken then is
restored; otherwise everything is recomputed inside the backward call.
"""
from __future__ import annotations

import torch

from . import pes


class PolyEval(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coeff, inputs, plan, memory_budget):
        value, _grad = plan.eval_grad(coeff, inputs)
        ctx.plan = plan
        ctx.generation = plan.generation
        ctx.snapshot = None
        if memory_budget is not None:
            nbytes = plan.info()["workspace_bytes"]
            if nbytes <= memory_budget:
                snap = torch.empty(nbytes, dtype=torch.uint8, device=coeff.device)
                plan.workspace_io(snap, to_buffer=True)
                ctx.snapshot = snap
        ctx.save_for_backward(coeff, inputs)
        return value

    @staticmethod
    def backward(ctx, grad_value):
        coeff, inputs = ctx.saved_tensors
        plan = ctx.plan
        u = grad_value.contiguous()
        if plan.generation == ctx.generation:
            reuse = True  # the workspace still holds this forward's products
        elif ctx.snapshot is not None:
            plan.workspace_io(ctx.snapshot, to_buffer=False)
            reuse = True
        else:
            reuse = False
        ctx.reused = reuse
        grad_inputs, grad_coeff = plan.vjp(coeff, inputs, u, reuse_forward=reuse)
        return grad_coeff, grad_inputs, None, None


def poly_eval(coeff, inputs, plan, memory_budget=None):
    """Value series of the polynomial of `plan` at `inputs`, differentiable with
    respect to `coeff` (k, N+1, d+1) and `inputs` (k, n, d+1).  With a
    pes.System the values are (k, P, d+1), one series per polynomial, and
    `coeff` is (k, N+P, d+1)."""
    if not isinstance(plan, pes.Plan):
        raise TypeError("plan must be a paper_2101_10881_gb300.pes.Plan")
    return PolyEval.apply(coeff, inputs, plan, memory_budget)
