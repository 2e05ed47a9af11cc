"""Masked-Galerkin closed form of the Smolyak operator (test infrastructure only).

A second, independent route to y = H_S x, valid when every 1D quadrature a
term uses is exact for the matrix elements it forms.  With the Hermite basis
and Gauss-Hermite grids this holds when, for every mode and every level,
    2*(nb(l)-1) + p <= 2*nq(l) - 1,
p being the largest per-mode degree of the Hamiltonian in that mode (2 for the
kinetic part).  Then each term's action is the Galerkin block P_l H P_l^T and
the combination of Eq. (16) collapses, by the identity
    sum_{l in R(l), l >= m} D_l = [ |m| <= L ]        (D_l of Eq. (8)),
to a masked matrix:
    (H_S)_{k k'} = [ sum_i lmin_i(max(k_i, k'_i)) <= L ] * <k|H|k'>,
where <k|H|k'> is the exact matrix element in the infinite Hermite basis,
built here from ladder operators (no quadrature at all).

Only the compact-basis order is shared with the C oracle (it is pinned on its
own by Table 2).
"""
from __future__ import annotations

import itertools

import numpy as np

from . import oracle as _orc


def _lmin(A: int, B: int, k: np.ndarray) -> np.ndarray:
    """smallest level whose basis holds index k: nb(l) = A + B l > k."""
    if B == 0:
        return np.where(k < A, 0, 10 ** 6)
    return np.maximum(0, -((A - 1 - k) // B))  # ceil((k+1-A)/B)


def _position_matrix(n: int, q0: float, s: float) -> np.ndarray:
    """Q = q0 + x/s in the Hermite basis, x = (a + a^dagger)/sqrt(2), truncated to n."""
    X = np.zeros((n, n))
    for k in range(n - 1):
        X[k, k + 1] = X[k + 1, k] = np.sqrt((k + 1) / 2.0)
    return q0 * np.eye(n) + X / s


def _d2_matrix(n: int, s: float) -> np.ndarray:
    """d^2/dQ^2 = s^2 d^2/dx^2, d/dx = (a - a^dagger)/sqrt(2), truncated to n."""
    P = np.zeros((n, n))
    for k in range(n - 1):
        # <k|d/dx|k+1> = sqrt((k+1)/2), <k+1|d/dx|k> = -sqrt((k+1)/2)
        P[k, k + 1] = np.sqrt((k + 1) / 2.0)
        P[k + 1, k] = -np.sqrt((k + 1) / 2.0)
    return s * s * (P @ P)


def exactness_violations(p):
    """List of (mode, level) where the quadrature is not exact for this Hamiltonian."""
    deg = np.zeros(p.D, int)
    off = 0
    for m in range(p.nmono):
        for f in range(off, off + int(p.nfac[m])):
            deg[p.fmode[f]] = max(deg[p.fmode[f]], int(p.fpow[f]))
        off += int(p.nfac[m])
    bad = []
    for i in range(p.D):
        d = max(deg[i], 2 if p.omega[i] != 0.0 else 0)
        for l in range(p.L + 1):
            nb = p.nb_A[i] + p.nb_B[i] * l
            nq = p.nq_A[i] + p.nq_B[i] * l
            if 2 * (nb - 1) + d > 2 * nq - 1:
                bad.append((i, l))
    return bad


def apply_H(p, x: np.ndarray) -> np.ndarray:
    """y = H_S x through the masked Galerkin matrix (raises if not exact)."""
    return _masked_galerkin(p, x=x)


def matrix(p):
    """The masked Galerkin matrix itself as scipy.sparse CSR (raises if not exact)."""
    return _masked_galerkin(p, x=None)


def _masked_galerkin(p, x=None):
    """Applies the masked Galerkin matrix to x, or (x None) assembles it."""
    bad = exactness_violations(p)
    if bad:
        raise ValueError(f"masked Galerkin form not exact for this problem: {bad[:4]}")
    D, L = p.D, p.L
    K = _orc.enumerate_compact(D, L, p.nb_A, p.nb_B).astype(np.int64)   # (N, D)
    N = K.shape[0]
    kmax = int(K.max()) if N else 0
    radix = kmax + 8
    weights = radix ** np.arange(D - 1, -1, -1, dtype=np.int64)
    keys = K @ weights            # lexicographic order == increasing key
    assert np.all(np.diff(keys) > 0)
    lm = np.stack([_lmin(int(p.nb_A[i]), int(p.nb_B[i]), K[:, i]) for i in range(D)], axis=1)

    assemble = x is None
    if assemble:
        parts = []   # (rows, cols, vals)
        X = Y = None
        squeeze = False
    else:
        x = np.asarray(x, np.float64)
        squeeze = x.ndim == 1
        X = x.reshape(1, -1) if squeeze else x
        Y = np.zeros_like(X)
    nmat = kmax + 8
    Qm = [_position_matrix(nmat + 4, float(p.q0[i]), float(p.scale[i])) for i in range(D)]
    D2m = [_d2_matrix(nmat + 4, float(p.scale[i])) for i in range(D)]

    def add_product(coef, ops):
        """ops: dict mode -> (n x n matrix, bandwidth)."""
        modes = sorted(ops)
        ranges = [range(-ops[i][1], ops[i][1] + 1) for i in modes]
        for shift in itertools.product(*ranges):
            Kp = K.copy()
            val = np.full(N, coef, np.float64)
            for i, d in zip(modes, shift):
                Kp[:, i] = K[:, i] + d
            ok = np.all(Kp >= 0, axis=1) & np.all(Kp <= kmax, axis=1)
            for i, d in zip(modes, shift):
                M = ops[i][0]
                kk = np.clip(K[:, i], 0, M.shape[0] - 1)
                kp = np.clip(Kp[:, i], 0, M.shape[0] - 1)
                val = val * M[kk, kp]
            # mask: sum_i lmin_i(max(k_i, k'_i)) <= L
            lsum = lm.sum(axis=1).copy()
            for i in modes:
                mx = np.maximum(K[:, i], Kp[:, i])
                lsum += _lmin(int(p.nb_A[i]), int(p.nb_B[i]), mx) - lm[:, i]
            ok &= lsum <= L
            ok &= val != 0.0
            if not np.any(ok):
                continue
            kp_keys = Kp[ok] @ weights
            pos = np.searchsorted(keys, kp_keys)
            found = (pos < N)
            pos_c = np.minimum(pos, N - 1)
            found &= keys[pos_c] == kp_keys
            rows = np.nonzero(ok)[0][found]
            cols = pos_c[found]
            if assemble:
                parts.append((rows, cols, val[rows]))
            else:
                Y[:, rows] += val[rows] * X[:, cols]

    off = 0
    for m in range(p.nmono):
        ops = {}
        for f in range(off, off + int(p.nfac[m])):
            i, pw = int(p.fmode[f]), int(p.fpow[f])
            M = np.linalg.matrix_power(Qm[i], pw) if i not in ops else ops[i][0] @ np.linalg.matrix_power(Qm[i], pw)
            bw = pw if i not in ops else ops[i][1] + pw
            ops[i] = (M, bw)
        off += int(p.nfac[m])
        if ops:
            add_product(float(p.coef[m]), ops)
        elif assemble:
            parts.append((np.arange(N), np.arange(N), np.full(N, float(p.coef[m]))))
        else:
            Y += float(p.coef[m]) * X
    for j in range(D):
        if p.omega[j] != 0.0:
            add_product(-0.5 * float(p.omega[j]), {j: (D2m[j], 2)})
    if assemble:
        import scipy.sparse as sp
        r = np.concatenate([a for a, _, _ in parts]) if parts else np.zeros(0, np.int64)
        c = np.concatenate([b for _, b, _ in parts]) if parts else np.zeros(0, np.int64)
        v = np.concatenate([w for _, _, w in parts]) if parts else np.zeros(0)
        return sp.csr_matrix((v, (r, c)), shape=(N, N))   # duplicates are summed
    return Y.reshape(-1) if squeeze else Y
