"""Dense Kronecker brute force of the Smolyak operator (test infrastructure only).

A third route to y = H_S x for tiny problems (D <= 3).  It shares nothing with
the C oracle's arithmetic: its own term enumeration (itertools), its own
compact basis and lookup, numpy's Gauss-Hermite rule, Hermite polynomials from
numpy's series evaluation and their derivatives from numpy's series
derivative, and dense Kronecker-product matrices on each term's full grid:

    H_S = sum_{l in R(l)} D_l  P_l^T (x_i B_i^T W_i)
          [ diag V(Q) (x_i B_i) + sum_j (-omega_j/2) (x_{i!=j} B_i x D2_j) ] P_l

(Eqs. (8), (14)-(16) with the grid operator written as a dense matrix.)
"""
from __future__ import annotations

import itertools
import math

import numpy as np
from numpy.polynomial import hermite as H


def hermite_functions_and_d2(nb: int, nq: int, q0: float, s: float):
    """B[u,k] = b_k(Q_u), D2[u,k] = b_k''(Q_u), W[u], Q[u] on the nq-point rule."""
    x, wg = H.hermgauss(nq)
    B = np.zeros((nq, nb)); D2 = np.zeros((nq, nb))
    g = np.exp(-0.5 * x * x)
    for k in range(nb):
        c = np.zeros(k + 1); c[k] = 1.0
        Nk = 1.0 / math.sqrt((2.0 ** k) * math.factorial(k) * math.sqrt(math.pi))
        Hk = H.hermval(x, c)
        dH = H.hermval(x, H.hermder(c, 1)) if k >= 1 else np.zeros_like(x)
        ddH = H.hermval(x, H.hermder(c, 2)) if k >= 2 else np.zeros_like(x)
        # (H e^{-x^2/2})'' = (H'' - 2x H' + (x^2 - 1) H) e^{-x^2/2}
        B[:, k] = math.sqrt(s) * Nk * Hk * g
        D2[:, k] = math.sqrt(s) * s * s * Nk * (ddH - 2 * x * dH + (x * x - 1) * Hk) * g
    W = wg * np.exp(x * x) / s
    Q = q0 + x / s
    return B, D2, W, Q


def dense_H(p) -> np.ndarray:
    D, L = p.D, p.L
    nb = lambda i, l: int(p.nb_A[i] + p.nb_B[i] * l)
    nq = lambda i, l: int(p.nq_A[i] + p.nq_B[i] * l)
    # compact basis: union of boxes, lexicographic, first mode slowest
    boxes = []
    terms = []
    for l in itertools.product(range(L + 1), repeat=D):
        s = sum(l)
        if L - D + 1 <= s <= L:
            terms.append(l)
    compact = set()
    for l in terms:
        for k in itertools.product(*[range(nb(i, l[i])) for i in range(D)]):
            compact.add(k)
    compact = sorted(compact)
    index = {k: n for n, k in enumerate(compact)}
    N = len(compact)
    HS = np.zeros((N, N))
    for l in terms:
        r = L - sum(l)
        c = (-1) ** r * math.comb(D - 1, r)
        tabs = [hermite_functions_and_d2(nb(i, l[i]), nq(i, l[i]), float(p.q0[i]), float(p.scale[i]))
                for i in range(D)]
        Bf = np.ones((1, 1)); BWf = np.ones((1, 1))
        for (B, D2, W, Q) in tabs:
            Bf = np.kron(Bf, B)
            BWf = np.kron(BWf, B.T * W[None, :])
        # grid coordinates (first mode slowest, as np.kron orders them)
        grids = np.meshgrid(*[t[3] for t in tabs], indexing="ij")
        V = np.zeros(grids[0].shape) if D else np.zeros(())
        off = 0
        for m in range(p.nmono):
            term = np.full(V.shape, float(p.coef[m]))
            for f in range(off, off + int(p.nfac[m])):
                term = term * grids[int(p.fmode[f])] ** int(p.fpow[f])
            V = V + term
            off += int(p.nfac[m])
        Og = np.diag(V.reshape(-1)) @ Bf
        for j in range(D):
            if p.omega[j] == 0.0:
                continue
            Kj = np.ones((1, 1))
            for i, (B, D2, W, Q) in enumerate(tabs):
                Kj = np.kron(Kj, D2 if i == j else B)
            Og = Og + (-0.5 * float(p.omega[j])) * Kj
        A = BWf @ Og
        box = list(itertools.product(*[range(nb(i, l[i])) for i in range(D)]))
        idx = np.array([index[k] for k in box])
        HS[np.ix_(idx, idx)] += c * A
    return HS


def apply_H(p, x: np.ndarray) -> np.ndarray:
    HS = dense_H(p)
    x = np.asarray(x, np.float64)
    return x @ HS.T if x.ndim == 2 else HS @ x
