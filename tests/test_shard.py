"""One polynomial split over ranks (host side, no GPU): the monomial split, the
rounding of digit sums on the host, and the exchange protocol with two gloo
ranks.

The addition stage sums the contributions of every output coefficient on the
largest grid among them -- each contribution's L digits shifted down to that
grid, digits falling below the L-th dropped -- and rounds the sum once.  Split
over ranks, the same sums come out of an integer all-reduce (maximum) of the
grids and an integer all-reduce (sum) of the digit sums: exact in any order.
These tests drive that protocol on synthetic digit-form contributions (random
digits and grids), two processes over gloo, and check that every rank rounds
bit for bit what one process computes from all contributions, and that the
rounded result is the exact sum within the k-double tolerance.
"""
import os
import socket
from fractions import Fraction

import numpy as np
import pytest

from paper_2101_10881_gb300 import pes, synth
from tests.exact import TOL

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
B = 28  # digit width of the integer pipe


@pytest.fixture(scope="module", autouse=True)
def built():
    pes.build()


def digits_of_k(k):
    return (53 * k + 28 + B - 1) // B + 1


def cost(s):
    return 3 * len(s) - 3 if len(s) >= 2 else 1


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_range_covers_and_balances(world):
    """Contiguous ranges, together every monomial once, each rank's jobs within
    one monomial of the even share."""
    rng = np.random.default_rng(world)
    for supports in (synth.supports_p2(), synth.random_supports(rng, 20, 57, 1, 9), [[0]], []):
        N = len(supports)
        ranges = [pes.shard_range(supports, world, r) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == N
        for (b0, e0), (b1, _) in zip(ranges, ranges[1:]):
            assert b0 <= e0 == b1
        W = sum(cost(s) for s in supports)
        biggest = max((cost(s) for s in supports), default=0)
        for b, e in ranges:
            assert sum(cost(s) for s in supports[b:e]) <= W / world + biggest


def test_shard_range_rejects_bad_arguments():
    for world, rank in ((0, 0), (2, 2), (2, -1)):
        with pytest.raises(pes.PesError):
            pes.shard_range([[0, 1]], world, rank)


def synthetic_contributions(rng, n_items, n_contrib, L):
    """Per item: a list of (grid, digits, factor) with balanced B-bit digits
    (leading digit nonzero) on grids within a few digits of each other, some
    far below (dropped), factors as the exponents of powers."""
    items = []
    for _ in range(n_items):
        cs = []
        base = int(rng.integers(-3, 4))
        for _ in range(n_contrib):
            g = base - int(rng.choice([0, 0, 0, 1, 2, 3, L + 2]))
            dg = rng.integers(-(1 << (B - 1)), 1 << (B - 1), size=L, dtype=np.int64)
            if dg[0] == 0:
                dg[0] = 1
            cs.append((g, dg, int(rng.choice([1, 1, 2, 3]))))
        items.append(cs)
    return items


def local_grids(items):
    return np.array([max(g for g, _, _ in cs) if cs else -(1 << 29) for cs in items], dtype=np.int32)


def local_sums(items, grids, L):
    """The addition stage's rule: every contribution's digits shifted down to
    the common grid, digits below the L-th dropped, summed exactly."""
    acc = np.zeros((len(items), L), dtype=np.int64)
    for it, cs in enumerate(items):
        for g, dg, mu in cs:
            sh = int(grids[it]) - g
            if sh >= L:
                continue
            for q in range(sh, L):
                acc[it, q] += mu * int(dg[q - sh])
    return acc


def exact_value(cs, L):
    """Exact sum of the contributions (all their digits)."""
    total = Fraction(0)
    for g, dg, mu in cs:
        for p in range(L):
            total += mu * Fraction(int(dg[p])) * Fraction(2) ** (B * (g - 1 - p))
    return total


def split_items(items, rank, world):
    """Contribution c of every item goes to rank c mod world."""
    return [[c for i, c in enumerate(cs) if i % world == rank] for cs in items]


def rank_main(rank, world, port, out_dir, k, n, d, seed):
    import json
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2101_10881_gb300 import pes as P

    L = digits_of_k(k)
    rng = np.random.default_rng(seed)
    items = synthetic_contributions(rng, (n + 1) * (d + 1), 5, L)
    mine = split_items(items, rank, world)
    grids = torch.from_numpy(local_grids(mine))
    dist.all_reduce(grids, op=dist.ReduceOp.MAX)
    acc = torch.from_numpy(local_sums(mine, grids.numpy(), L))
    dist.all_reduce(acc, op=dist.ReduceOp.SUM)
    value, grad = P.round_sums_host(k, n, d, grids.numpy().reshape(n + 1, d + 1),
                                    acc.numpy().reshape(n + 1, d + 1, L))
    np.save(os.path.join(out_dir, f"v{rank}.npy"), value)
    np.save(os.path.join(out_dir, f"g{rank}.npy"), grad)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"rank": rank}, f)
    dist.destroy_process_group()


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("k", [2, 10])
def test_exchange_two_gloo_ranks_bit_identical(k, tmp_path):
    n, d, seed, world = 3, 6, 11 + k, 2
    mp.start_processes(rank_main, args=(world, free_port(), str(tmp_path), k, n, d, seed), nprocs=world, join=True,
                       start_method="spawn")
    L = digits_of_k(k)
    items = synthetic_contributions(np.random.default_rng(seed), (n + 1) * (d + 1), 5, L)
    grids = local_grids(items)
    acc = local_sums(items, grids, L)
    v1, g1 = pes.round_sums_host(k, n, d, grids.reshape(n + 1, d + 1), acc.reshape(n + 1, d + 1, L))
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / f"v{r}.npy"), v1)
        assert np.array_equal(np.load(tmp_path / f"g{r}.npy"), g1)
    # the rounded sums are the exact sums of the kept digits, within the
    # k-double tolerance of the exact sum of every digit per output series
    out = np.concatenate([v1[:, None, :], g1], axis=1)  # (k, n+1, d+1)
    for o in range(n + 1):
        got = [sum(Fraction(float(x)) for x in out[:, o, j]) for j in range(d + 1)]
        ref = [exact_value(items[o * (d + 1) + j], L) for j in range(d + 1)]
        den = max(abs(r) for r in ref)
        assert max(abs(a - b) for a, b in zip(got, ref)) <= Fraction(TOL[k]) * den


def test_round_sums_host_is_the_nearest_limbs():
    """A digit sum with a known exact value rounds to the limbs of that value
    (each limb the nearest double of the remainder)."""
    k, n, d = 4, 1, 2
    L = digits_of_k(k)
    rng = np.random.default_rng(3)
    grids = np.array([[1, 0, -2], [2, 1, 0]], dtype=np.int32)
    acc = rng.integers(-(1 << 40), 1 << 40, size=(n + 1, d + 1, L), dtype=np.int64)
    v, g = pes.round_sums_host(k, n, d, grids, acc)
    out = np.concatenate([v[:, None, :], g], axis=1)
    for o in range(n + 1):
        for j in range(d + 1):
            exact = sum(Fraction(int(acc[o, j, p])) * Fraction(2) ** (B * (int(grids[o, j]) - 1 - p))
                        for p in range(L))
            assert list(out[:, o, j]) == synth.round_fraction_to_limbs(exact, k)
