"""One polynomial split over ranks by monomials (one GPU per rank).

The monomials are independent through the convolution layers (Sec. 5); only
the addition jobs combine their contributions.  Every rank plans the
polynomial of its own monomials (pes_shard_range: contiguous ranges balanced by
convolution jobs, the constant a_0 on rank 0), and the ranks exchange two
integer arrays through torch.distributed: the largest grid of every output
coefficient (all-reduce, maximum) and the exact digit sums on those grids
(all-reduce, sum).  Both are exact in any order, so every rank rounds the
same sums once and obtains, bit for bit, what one plan of the whole
polynomial gives.  A floating-point all-reduce of the rounded k-double limbs
would not be exact.

Argument marshalling and collectives only: the products, sums and rounding run
in libpes's kernels (include/pes.h, pes_partial_grids / pes_partial_sums /
pes_round_sums).
"""
from __future__ import annotations

import numpy as np

from . import pes


class ShardPlan:
    """The part of a polynomial that rank `rank` of `world` evaluates."""

    def __init__(self, supports, n, d, k, world, rank, exponents=None, **opts):
        self.world, self.rank = int(world), int(rank)
        self.m_begin, self.m_end = pes.shard_range(supports, world, rank)
        self.supports = [list(s) for s in supports[self.m_begin:self.m_end]]
        ex = None if exponents is None else [list(e) for e in exponents[self.m_begin:self.m_end]]
        self.n, self.d, self.k = int(n), int(d), int(k)
        self.plan = pes.Plan(self.supports, n, d, k, exponents=ex, with_vjp=False, **opts)

    def coeff_of(self, coeff):
        """This rank's coefficient buffer (k, N_r + 1, d+1) from the whole
        polynomial's (k, N + 1, d+1): a_0 on rank 0, zero on the others."""
        import torch
        part = coeff[:, 1 + self.m_begin:1 + self.m_end]
        a0 = coeff[:, :1] if self.rank == 0 else torch.zeros_like(coeff[:, :1])
        return torch.cat([a0, part], dim=1).contiguous()

    def eval_grad(self, coeff_r, inputs, group=None):
        """Value and gradient of the whole polynomial on every rank of `group`
        (torch.distributed, one GPU per rank); coeff_r from coeff_of."""
        import torch.distributed as dist
        grids = self.plan.partial_grids(coeff_r, inputs)
        if self.world > 1:
            dist.all_reduce(grids, op=dist.ReduceOp.MAX, group=group)
        acc = self.plan.partial_sums(grids)
        if self.world > 1:
            dist.all_reduce(acc, op=dist.ReduceOp.SUM, group=group)
        return self.plan.round_sums(grids, acc)


def combine_host(k, n, d, parts, arith="int"):
    """The exchange on the host, for (grids, acc) numpy pairs of every rank
    taken on common grids: sum the integer digit sums and round once
    (pes_round_sums_host)."""
    grids = parts[0][0]
    acc = np.zeros_like(parts[0][1])
    for g, a in parts:
        assert np.array_equal(g, grids)
        acc += a
    return pes.round_sums_host(k, n, d, grids, acc, arith=arith)
