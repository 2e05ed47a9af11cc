"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test compares the oracle with something other than itself:
  - values printed in the paper (Table 1, Table 2, the Fig. 1 description);
  - library routines for special cases (numpy's Gauss-Hermite rule);
  - closed forms (partition of unity of the combination technique, the
    separable-oscillator spectrum at zero coupling, the masked-Galerkin form);
  - an independent dense brute force on tiny problems;
  - invariants (Hermiticity).
"""
import math
import os

import numpy as np
import pytest

from oracle import bruteforce, galerkin
from oracle import oracle as orc
from paper_2111_13655_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _read_sections(path):
    sec, out = None, {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("["):
            sec = line.strip("[]")
            out[sec] = []
            continue
        out[sec].append(line.split())
    return out


# ---------------------------------------------------------------- Table 2 / Fig. 1
def test_table2_term_order_and_mapping():
    g = _read_sections(os.path.join(GOLDEN, "table2_mapping.txt"))
    lv, _ = orc.enumerate_terms(2, 3)
    off, cs = orc.term_map(2, 3)
    assert lv.shape[0] == len(g["terms"])
    for t, row in enumerate(g["terms"]):
        ist, l1, l2, *ics = map(int, row)
        assert ist == t + 1
        assert tuple(lv[t]) == (l1, l2)
        assert (cs[off[t]:off[t + 1]] + 1).tolist() == ics


def test_table2_compact_basis():
    g = _read_sections(os.path.join(GOLDEN, "table2_mapping.txt"))
    K = orc.enumerate_compact(2, 3)
    assert K.shape[0] == len(g["compact"])
    for row in g["compact"]:
        ics, k1, k2 = map(int, row)
        assert tuple(K[ics - 1]) == (k1, k2)


def test_fig1_counts():
    g = _read_sections(os.path.join(GOLDEN, "table2_mapping.txt"))
    facts = {r[0]: int(r[1]) for r in g["facts"]}
    nt, ns, ncs = orc.counts(2, 3)
    assert (nt, ns, ncs) == (facts["n_terms"], facts["n_s"], facts["n_cs"])
    off, cs = orc.term_map(2, 3)
    assert off[-1] == facts["n_s"] and len(set(cs.tolist())) == facts["n_cs"]


# ---------------------------------------------------------------- Table 1
def test_table1_counts():
    for line in open(os.path.join(GOLDEN, "table1_counts.txt")):
        if line.startswith("#") or not line.strip():
            continue
        D, L, ns, ncs, ratio = line.split()
        D, L, ns, ncs = int(D), int(L), int(ns), int(ncs)
        nt, ns_o, ncs_o = orc.counts(D, L)
        assert (ns_o, ncs_o) == (ns, ncs), (D, L)
        assert f"{ns_o / ncs_o:.2f}" == ratio


@pytest.mark.parametrize("D,L,nbA,nbB", [(3, 4, 1, 1), (4, 3, 1, 2), (12, 3, 1, 1), (5, 4, 2, 1)])
def test_counts_match_enumeration(D, L, nbA, nbB):
    nt, ns, ncs = orc.counts(D, L, nbA, nbB)
    lv, c = orc.enumerate_terms(D, L)
    assert lv.shape[0] == nt
    off, cs = orc.term_map(D, L, nbA, nbB)
    assert off[-1] == ns
    K = orc.enumerate_compact(D, L, nbA, nbB)
    assert K.shape[0] == ncs == len(np.unique(cs))
    # compact list is sorted lexicographically with the first mode slowest, no duplicates
    keys = [tuple(k) for k in K]
    assert keys == sorted(set(keys))


def test_combination_coefficients_enumeration_order():
    # every term lies in R(l); l_1 varies fastest (Table 2 order)
    D, L = 4, 5
    lv, c = orc.enumerate_terms(D, L)
    s = lv.sum(1)
    assert np.all((s >= L - D + 1) & (s <= L))
    colex = [tuple(r[::-1]) for r in lv]
    assert colex == sorted(colex)
    assert len(set(map(tuple, lv))) == lv.shape[0]


# ---------------------------------------------------------------- 1D tables
@pytest.mark.parametrize("n", list(range(1, 21)))
def test_gauss_hermite_matches_library(n):
    x, w = orc.gauss_hermite(n)
    xr, wr = np.polynomial.hermite.hermgauss(n)
    assert np.allclose(x, xr, rtol=0, atol=1e-13 * max(1, abs(xr).max()))
    assert np.allclose(w, wr, rtol=1e-11, atol=1e-300)
    assert abs(w.sum() - math.sqrt(math.pi)) < 1e-13
    assert np.allclose(x, -x[::-1], atol=1e-13)


@pytest.mark.parametrize("nb,nq", [(1, 1), (1, 2), (3, 3), (4, 6), (11, 12), (7, 13)])
def test_basis_orthonormal_on_grid(nb, nq):
    B, D2, W, Q = orc.mode_tables(nb, nq, 0.3, 1.4)
    G = B.T @ (W[:, None] * B)
    assert np.abs(G - np.eye(nb)).max() < 1e-13


@pytest.mark.parametrize("nb,nq,q0,s", [(4, 5, 0.0, 1.0), (6, 6, -0.4, 0.7), (3, 9, 1.0, 2.0)])
def test_mode_tables_match_independent_evaluation(nb, nq, q0, s):
    B, D2, W, Q = orc.mode_tables(nb, nq, q0, s)
    B2, D22, W2, Q2 = bruteforce.hermite_functions_and_d2(nb, nq, q0, s)
    assert np.abs(B - B2).max() < 1e-12
    assert np.abs(D2 - D22).max() < 1e-10 * max(1, np.abs(D22).max())
    assert np.allclose(W, W2, rtol=1e-11)
    assert np.allclose(Q, Q2, atol=1e-12)


# ---------------------------------------------------------------- operator action
@pytest.mark.parametrize("D,L,nq_rule,nb_rule", [
    (1, 4, (1, 1), (1, 1)), (2, 3, (1, 1), (1, 1)), (3, 4, (2, 1), (1, 1)),
    (4, 5, (1, 2), (1, 1)), (6, 3, (1, 1), (1, 1)), (3, 3, (3, 2), (1, 2))])
def test_partition_of_unity(D, L, nq_rule, nb_rule):
    """V = 1, no kinetic part: sum_l D_l P_l^T P_l = identity on the compact basis."""
    p = synth.polynomial_problem(D, L, np.zeros(D), [(1.0, [])], nb_rule=nb_rule, nq_rule=nq_rule)
    n = orc.n_compact(p)
    x = synth.random_vectors(n, 2, 11)
    assert rel(orc.apply_H(p, x), x) < 1e-13


@pytest.mark.parametrize("D,L,nq_rule", [(2, 6, (1, 1)), (3, 5, (1, 1)), (4, 4, (2, 1)), (6, 3, (1, 2))])
def test_uncoupled_oscillators_are_diagonal(D, L, nq_rule):
    """lambda = 0: H_S |k> = sum_i omega_i (k_i + 1/2) |k> for any nq >= nb."""
    om = synth.draw_omega(D, 21)
    p = synth.chained_henon_heiles(D, L, om, 0.0, nq_rule=nq_rule)
    K = orc.enumerate_compact(D, L)
    E = (K + 0.5) @ om
    x = synth.random_vectors(K.shape[0], 2, 5)
    assert rel(orc.apply_H(p, x), E[None, :] * x) < 1e-13


@pytest.mark.parametrize("D,L,lam", [(2, 5, 0.111803), (3, 4, 0.3), (4, 5, 0.2), (6, 4, 0.111803)])
def test_masked_galerkin_closed_form(D, L, lam):
    """nq = l + 2 makes every term's quadrature exact for Henon-Heiles, so H_S is
    the masked Galerkin matrix built from ladder operators."""
    p = synth.chained_henon_heiles(D, L, synth.draw_omega(D, 31), lam, nq_rule=(2, 1))
    n = orc.n_compact(p)
    x = synth.random_vectors(n, 2, 7)
    assert rel(orc.apply_H(p, x), galerkin.apply_H(p, x)) < 1e-13


def test_masked_galerkin_detects_inexact_quadrature():
    """With nq = l + 1 the quadrature is not exact and the two routes must differ
    (the closed form refuses; forced comparison shows an O(1e-2) gap)."""
    p = synth.chained_henon_heiles(3, 4, [1.0, 1.0, 1.0], 0.3, nq_rule=(1, 1))
    assert galerkin.exactness_violations(p)
    with pytest.raises(ValueError):
        galerkin.apply_H(p, np.zeros(orc.n_compact(p)))


@pytest.mark.parametrize("D,L,nq_rule", [(1, 6, (1, 1)), (2, 6, (1, 1)), (2, 4, (1, 2)), (3, 4, (1, 1))])
def test_dense_brute_force(D, L, nq_rule):
    p = synth.chained_henon_heiles(D, L, synth.draw_omega(D, 41), 0.3, nq_rule=nq_rule)
    n = orc.n_compact(p)
    x = synth.random_vectors(n, 3, 9)
    assert rel(orc.apply_H(p, x), bruteforce.apply_H(p, x)) < 1e-13


def test_dense_brute_force_general_polynomial_shifted_scaled():
    monos = [(0.3, [(0, 1)]), (0.2, [(0, 2), (1, 2)]), (-0.1, [(1, 3)]), (0.05, [(0, 1), (1, 1)]),
             (0.7, [])]
    p = synth.polynomial_problem(2, 4, [0.9, 1.1], monos, q0=[0.3, -0.2], scale=[1.3, 0.8])
    n = orc.n_compact(p)
    x = synth.random_vectors(n, 2, 3)
    assert rel(orc.apply_H(p, x), bruteforce.apply_H(p, x)) < 1e-13


@pytest.mark.parametrize("D,L,nq_rule", [(3, 5, (1, 1)), (5, 4, (1, 1)), (4, 4, (1, 2))])
def test_hermitian(D, L, nq_rule):
    p = synth.chained_henon_heiles(D, L, synth.draw_omega(D, 51), 0.111803, nq_rule=nq_rule)
    n = orc.n_compact(p)
    x = synth.random_vectors(n, 2, 13)
    y = orc.apply_H(p, x)
    a, b = x[0] @ y[1], y[0] @ x[1]
    assert abs(a - b) < 1e-13 * (np.linalg.norm(y[0]) + np.linalg.norm(y[1]))


def test_term_subset_sums_to_full():
    p = synth.chained_henon_heiles(4, 5, synth.draw_omega(4, 61), 0.2)
    n = orc.n_compact(p)
    x = synth.random_vectors(n, 1, 1)
    nt = orc.counts(4, 5)[0]
    idx = np.arange(nt)
    y = orc.apply_H(p, x, idx[::2]) + orc.apply_H(p, x, idx[1::2])
    assert rel(y, orc.apply_H(p, x)) < 1e-14


def test_thread_count_does_not_change_result_beyond_rounding():
    p = synth.chained_henon_heiles(4, 5, synth.draw_omega(4, 71), 0.2)
    n = orc.n_compact(p)
    x = synth.random_vectors(n, 1, 1)
    assert rel(orc.apply_H(p, x, threads=1), orc.apply_H(p, x, threads=3)) < 1e-14


def test_masked_galerkin_matrix_is_its_apply_and_symmetric():
    """The assembled masked-Galerkin matrix (used for the stored D=12 L=10
    eigenvalues) is the same operator as its apply path, and symmetric (P8)."""
    from oracle import galerkin
    p = synth.workload_C3(L=4, D=5)
    M = galerkin.matrix(p)
    x = np.random.default_rng(3).standard_normal((2, M.shape[0]))
    y = galerkin.apply_H(p, x)
    assert np.abs((M @ x.T).T - y).max() <= 1e-13 * np.abs(y).max()
    assert abs(M - M.T).max() <= 1e-14


# ---------------------------------------------------------------- Smolyak quadrature exactness

def _hermite_function(k, q):
    """Orthonormal Hermite function b_k(q), through numpy's physicists' Hermite series."""
    c = np.zeros(k + 1)
    c[k] = 1.0
    norm = math.sqrt(2.0 ** k * math.factorial(k) * math.sqrt(math.pi))
    return np.polynomial.hermite.hermval(q, c) * np.exp(-q * q / 2) / norm


def _gaussian_moment(p):
    """int b_0(q)^2 q^p dq = (p-1)!!/2^(p/2) for even p, 0 for odd p."""
    if p % 2:
        return 0.0
    return math.prod(range(p - 1, 0, -2)) / 2.0 ** (p // 2)


def _surplus_column(D, L, nb_rule, nq_rule, monos):
    """Column H_S e_0 of a kinetic-free problem with V = sum of product monomials,
    from the hierarchical (surplus) form of the Smolyak formula instead of the
    combination coefficients: sum_{|l| <= L} prod_i (g_i(l_i) - g_i(l_i - 1)),
    where g_i(l) = [k_i < nb(l)] sum_u w_u b_{k_i}(Q_u) b_0(Q_u) Q_u^{p_i} on
    numpy's level-l Gauss-Hermite rule (weights times e^{Q^2}, so that the rule
    integrates b_k b_k' exactly).  The combination formula of Eq. (8) and this
    hierarchical form are the same sum for any per-mode sequences g_i (an identity
    of the combination technique); the 1D rules enter through Eqs. (6)-(7)."""
    import itertools

    nb = lambda l: nb_rule[0] + nb_rule[1] * l
    nq = lambda l: nq_rule[0] + nq_rule[1] * l
    lmin = lambda k: next(l for l in range(L + 1) if nb(l) > k)
    compact = [k for k in itertools.product(range(nb(L)), repeat=D) if sum(lmin(ki) for ki in k) <= L]

    def g(l, k, p):
        if l < 0 or k >= nb(l):
            return 0.0
        x, w = np.polynomial.hermite.hermgauss(nq(l))
        return float(np.sum(w * np.exp(x * x) * _hermite_function(k, x) * _hermite_function(0, x) * x ** p))

    levels = [l for l in itertools.product(range(L + 1), repeat=D) if sum(l) <= L]
    y = np.zeros(len(compact))
    for c, factors in monos:
        pw = [0] * D
        for mode, power in factors:
            pw[mode] = power
        for j, k in enumerate(compact):
            y[j] += c * sum(math.prod(g(l[i], k[i], pw[i]) - g(l[i] - 1, k[i], pw[i]) for i in range(D))
                            for l in levels)
    return y


@pytest.mark.parametrize("D, L, nq_rule, monos", [
    (2, 3, (1, 1), [(1.0, [(0, 4), (1, 2)])]),
    (2, 2, (1, 1), [(1.0, [(0, 4), (1, 2)])]),                        # not exact at this level
    (3, 4, (1, 1), [(0.7, [(0, 3), (2, 2)]), (1.3, [(1, 2)])]),
    (2, 5, (1, 2), [(1.0, [(0, 5), (1, 1)]), (-0.4, [(0, 2), (1, 6)])]),
])
def test_smolyak_quadrature_of_monomials(D, L, nq_rule, monos):
    """Kinetic-free V = sum of monomials, ground state in: the oracle's column equals
    the hierarchical Smolyak sum; <0|H_S|0> is the exact Gaussian moment product
    exactly when levels e(p_i) with 2 nq(e) - 1 >= p_i fit within L (Smolyak
    quadrature exactness), and differs from it otherwise."""
    p = synth.polynomial_problem(D, L, np.zeros(D), monos, nb_rule=(1, 1), nq_rule=nq_rule)
    n = orc.n_compact(p)
    x = np.zeros((1, n))
    x[0, 0] = 1.0
    y = orc.apply_H(p, x)[0]
    ref = _surplus_column(D, L, (1, 1), nq_rule, monos)
    assert y.shape == ref.shape
    assert np.abs(y - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())
    exact, within = 0.0, True
    for c, factors in monos:
        exact += c * math.prod(_gaussian_moment(pw) for _, pw in factors)
        e = [next(l for l in range(100) if 2 * (nq_rule[0] + nq_rule[1] * l) - 1 >= pw) for _, pw in factors]
        within &= sum(e) <= L
    if within:
        assert abs(y[0] - exact) <= 1e-13 * max(1.0, abs(exact))
    else:
        assert abs(y[0] - exact) > 1e-6
