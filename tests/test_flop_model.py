"""The algorithmic FLOP count behind bench.py's roofline figure, checked on the CPU.

F_alg must describe the route the kernel takes: per term, the forward chain
of one-mode contractions over the modes with nb > 1 in the order the host
plans (ascending 1/nb - 1/nq, ties in mode order), the mirrored backward
chain, the basis-part matrices, one multiply per grid point and the
compress-add.  Two checks: the vectorised count equals a per-term loop, and
the planned order is the cheapest of all orders (brute force over
permutations), which is what the swap argument for that order claims.
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
    act = [l for l in levels if nbA + nbB * l > 1]
    nbs = [nbA + nbB * l for l in act]
    nqs = [nqA + nqB * l for l in act]
    order = planned_order(nbs, nqs)
    fwd = chain_fmas([nbs[j] for j in order], [nqs[j] for j in order])
    NB, NG = math.prod(nbs), math.prod(nqs)
    kin = NB * sum(nbs)
    return 2 * (2 * fwd + kin) + NG + 2 * NB


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
    """D=12 L=10, nb = l+1, nq = l+2: 3.70e10 FLOPs per vector in the planned
    order (the figure the benchmark's roofline uses)."""
    from oracle import oracle as orc
    lv, _ = orc.enumerate_terms(12, 10)
    f = bench.algorithmic_flops_per_vector(np.asarray(lv))
    assert f == 37029384645
