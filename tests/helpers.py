"""Error measures and tolerances of the GPU parity tests, and a cached dense
oracle matrix for the propagation checks.

Two measures, both per vector, the worst vector reported:
  norm_rel(y, r) = ||y - r||_2 / ||r||_2
  elem_rel(y, r) = max_i |y_i - r_i| / max_i |r_i|
The element-wise form catches a single wrong entry (a mis-ranked compact
index, a dropped or doubled term) that the 2-norm would dilute by up to
sqrt(N_cs).

FP64 mode: both <= 1e-12 against an exact reference (the masked-Galerkin
closed form where it applies).  The literal oracle sums the terms' D_l y_l in
floating point; at the compact function k = 0, which every term touches, its
own rounding reaches u * sum_l |D_l| * max|y_l| (u = 2^-53): 3.3e-12 of
max|y| at D=12 L=5 against the closed form, measured.  Element-wise
comparisons with the literal oracle therefore allow max(1e-12, u sum_l |D_l|)
(literal_elem_tol); norm-wise stays 1e-12.
Mixed mode (FP32 contractions, exact fixed-point sum): every term's result
carries FP32 rounding (~6e-8 relative) and the combination coefficients D_l
(Eq. (8); |D_l| up to 462 at D=12) sum those errors over the terms sharing a
compact function.  The compact function k = 0 lies in every term, so its
error is the largest: the element-wise measure is looser than the norm-wise
one.  Measured on GB300 (mixed vs the oracle): element-wise 1.1e-8 (D=2 L=6),
2.0e-7 (D=6 L=8), 3.0e-7 (D=12 L=5), 1.4e-7 (general polynomial); norm-wise
at most 1.2e-7.  MIXED_ELEM_TOL = 5e-6 keeps a margin above 15 over them.
Double-float mode (SG_DF64: each contraction value a pair of FP32 numbers,
about 48 significant bits, exact fixed-point sum): every term's result
carries a relative rounding of a few u_df = 2^-48 per operation (against
2^-53 in FP64; tests/test_df_arith.py pins the operations' bounds), 32 times
FP64's, and the compact functions shared by many terms collect it with the
weights |D_l| as in mixed mode.  Norm-wise the FP64 bound 1e-12 holds (measured
on GB300 against the exact closed form: 1.3e-15 at D=12 L=5, 8.7e-14 at
D=12 L=10); element-wise the measure reaches 1.7e-14 at D=12 L=5 and 3.6e-12
at D=12 L=10, so DF64_ELEM_TOL = 1e-11 (a margin near three over the largest).
"""
import numpy as np

FP64_TOL = 1e-12
MIXED_TOL = 5e-6
MIXED_ELEM_TOL = 5e-6
DF64_TOL = 1e-12
DF64_ELEM_TOL = 1e-11


def literal_elem_tol(p):
    """Element-wise FP64 tolerance against the literal oracle: its own
    floating-point compress-add bound u * sum_l |D_l| (Eq. (8)), at least 1e-12."""
    from oracle import oracle as orc
    _, c = orc.enumerate_terms(p.D, p.L)
    return max(FP64_TOL, 2.0 ** -53 * float(np.abs(np.asarray(c, float)).sum()))


def norm_rel(y, r):
    y = np.atleast_2d(y); r = np.atleast_2d(r)
    return float(np.max(np.linalg.norm(y - r, axis=1) / np.linalg.norm(r, axis=1)))


def elem_rel(y, r):
    y = np.atleast_2d(y); r = np.atleast_2d(r)
    return float(np.max(np.max(np.abs(y - r), axis=1) / np.max(np.abs(r), axis=1)))


def assert_parity(y, r, precision, what=""):
    """Both measures within the tolerances of `precision` ("fp64", "df64" or "mixed")."""
    n, e = norm_rel(y, r), elem_rel(y, r)
    if precision == "fp64":
        assert n <= FP64_TOL and e <= FP64_TOL, f"{what}: norm-wise {n:.3e}, element-wise {e:.3e}"
    elif precision == "df64":
        assert n <= DF64_TOL and e <= DF64_ELEM_TOL, f"{what}: norm-wise {n:.3e}, element-wise {e:.3e}"
    else:
        assert n <= MIXED_TOL and e <= MIXED_ELEM_TOL, f"{what}: norm-wise {n:.3e}, element-wise {e:.3e}"
    return n, e


_DENSE = {}


def dense_oracle(p):
    """H_S of problem p as a dense symmetric matrix, column j = H_S e_j, from
    the literal CPU oracle (symmetrised: H_S is symmetric, Sec. 2); cached per
    problem name within a test process."""
    from oracle import oracle as orc
    key = (p.name, p.D, p.L, tuple(np.asarray(p.omega).round(15)), tuple(np.asarray(p.coef).round(15)))
    if key not in _DENSE:
        n = orc.n_compact(p)
        H = orc.apply_H(p, np.eye(n)).T
        _DENSE[key] = 0.5 * (H + H.T)
    return _DENSE[key]


def exact_propagator(H):
    """(w, U) with H = U diag(w) U^T, for psi(t) = U exp(-i w t) U^T psi(0)."""
    return np.linalg.eigh(H)
