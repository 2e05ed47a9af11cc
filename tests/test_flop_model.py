"""The algorithmic FLOP count behind bench.py's roofline figure, checked on the CPU.

F_alg must describe the route the kernel takes: per term with a grid (two
neighbouring modes of the chain both transformed), the last three level-1
modes are inner positions whose block is applied at every outer grid point;
the forward chain of one-mode contractions over the other modes with nb > 1
runs in the order the host plans (ascending 1/nb - 1/nq, ties in mode order)
on NBI values per site, the backward chain mirrors it; then the single-mode
matrices of the outer modes and the compress-add.  Two checks: the vectorised
count equals a per-term loop, and the planned order is the cheapest of all
orders (brute force over permutations), which is what the swap argument for
that order claims.
"""
import itertools
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def chain_fmas(nbs, nqs):
    """Multiply-adds of the forward chain basis -> grid in the given order."""
    total = 0
    for j in range(len(nbs)):
        total += math.prod(nqs[:j]) * nbs[j] * nqs[j] * math.prod(nbs[j + 1:])
    return total


def planned_order(nbs, nqs):
    return sorted(range(len(nbs)), key=lambda j: (1.0 / nbs[j] - 1.0 / nqs[j], j))


def term_flops(levels, rule):
    nbA, nbB, nqA, nqB = rule
    nb1 = nbA + nbB
    rmax = 3 if nb1 == 2 else 2 if nb1 == 3 else 0
    D = len(levels)
    active = [nbA + nbB * l > 1 for l in levels]
    grid = any(active[i] and active[i + 1] for i in range(D - 1))
    inner = set()
    if grid:
        for i in range(D - 1, -1, -1):
            if len(inner) < rmax and levels[i] == 1 and active[i]:
                inner.add(i)
    outer = [i for i in range(D) if active[i] and i not in inner]
    nbs = [nbA + nbB * levels[i] for i in outer]
    nqs = [nqA + nqB * levels[i] for i in outer]
    NBI = math.prod(nbA + nbB * levels[i] for i in inner)
    order = planned_order(nbs, nqs)
    fwd = chain_fmas([nbs[j] for j in order], [nqs[j] for j in order]) * NBI
    NB = NBI * math.prod(nbs)
    reg = math.prod(nqs) * NBI * NBI if grid else 0
    basis = NB * (sum(nbs) + (0 if grid else 1))
    return 2 * (2 * fwd + reg + basis) + 2 * NB


@pytest.mark.parametrize("rule", [(1, 1, 2, 1), (1, 1, 1, 1), (2, 1, 3, 1), (1, 2, 1, 2)])
def test_vectorised_count_equals_per_term_loop(rule):
    rng = np.random.default_rng(5)
    levels = rng.integers(0, 5, size=(300, 7))
    ref = sum(term_flops(list(r), rule) for r in levels)
    assert bench.algorithmic_flops_per_vector(levels, *rule) == ref


@pytest.mark.parametrize("rule", [(1, 1, 2, 1), (2, 1, 3, 1), (1, 2, 2, 2)])
def test_planned_order_is_the_cheapest(rule):
    nbA, nbB, nqA, nqB = rule
    rng = np.random.default_rng(11)
    for _ in range(60):
        lv = [int(v) for v in rng.integers(1, 5, size=int(rng.integers(2, 6)))]
        nbs = [nbA + nbB * l for l in lv]
        nqs = [nqA + nqB * l for l in lv]
        order = planned_order(nbs, nqs)
        best = min(chain_fmas([nbs[j] for j in p], [nqs[j] for j in p])
                   for p in itertools.permutations(range(len(lv))))
        assert chain_fmas([nbs[j] for j in order], [nqs[j] for j in order]) == best


def test_benchmark_workload_count():
    """D=12 L=10, nb = l+1, nq = l+2: 1.97e10 FLOPs per vector by the kernel's
    route (the figure the benchmark's roofline uses)."""
    from oracle import oracle as orc
    lv, _ = orc.enumerate_terms(12, 10)
    f = bench.algorithmic_flops_per_vector(np.asarray(lv))
    assert f == 19703308878
