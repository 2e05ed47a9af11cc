"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module holds input *definitions* only: the Hamiltonian's parameters (a
sparse polynomial potential and per-mode kinetic prefactors), the per-mode
level -> size rules, and seeded random numbers.  It performs none of the
Smolyak arithmetic (no term enumeration, no quadrature, no index maps), so the
oracle and the GPU library can both be fed from it without sharing any of the
method's code.

Workload family (the paper's Sec. 4 example, Eq. (18), generalised to a chain):
    H = sum_i omega_i/2 * (-d^2/dq_i^2) + V(q),
    V = sum_i omega_i/2 * q_i^2 + lam * sum_{i<D} (q_i^2 q_{i+1} - q_{i+1}^3 / 3).
With omega_i = 1 this is exactly the Henon-Heiles Hamiltonian of Eq. (18).

Random numbers come from numpy's PCG64 generator seeded explicitly, so every
run (and both sides of a parity test) sees identical inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence

import numpy as np

# Coupling constant of the Henon-Heiles workloads (the literal value used by
# the benchmark configurations; sqrt(0.0125) to six digits).
HH_LAMBDA = 0.111803


@dataclass
class Problem:
    """A Smolyak operator-action problem: sizes, per-mode rules, Hamiltonian.

    Per-mode level->size rules follow Sec. 2 (N_l = A + B*l): basis size
    nb(l) = nb_A + nb_B*l and grid size nq(l) = nq_A + nq_B*l.  The primitive
    basis of every mode is the Hermite-function basis ("Hm", Sec. 4) centred
    at q0 with scale factor `scale`.

    The potential is a sparse polynomial: monomial m contributes
    coef[m] * prod_f q_{fmode[f]}^{fpow[f]} over its nfac[m] factors, the
    factors of all monomials being stored back to back in fmode/fpow.
    """

    D: int
    L: int
    nb_A: np.ndarray
    nb_B: np.ndarray
    nq_A: np.ndarray
    nq_B: np.ndarray
    q0: np.ndarray
    scale: np.ndarray
    omega: np.ndarray          # kinetic prefactor: T = sum_i omega_i/2 (-d^2/dq_i^2)
    coef: np.ndarray           # (nmono,) float64
    nfac: np.ndarray           # (nmono,) int32
    fmode: np.ndarray          # (sum nfac,) int32, 0-based mode index
    fpow: np.ndarray           # (sum nfac,) int32, power >= 1
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nmono(self) -> int:
        return int(self.coef.shape[0])


def _poly(monos: Sequence[tuple]) -> tuple:
    """monos: sequence of (coef, [(mode, power), ...])."""
    coef, nfac, fmode, fpow = [], [], [], []
    for c, facs in monos:
        coef.append(float(c))
        nfac.append(len(facs))
        for m, p in facs:
            fmode.append(int(m))
            fpow.append(int(p))
    return (np.asarray(coef, np.float64), np.asarray(nfac, np.int32),
            np.asarray(fmode, np.int32), np.asarray(fpow, np.int32))


def chained_henon_heiles(D: int, L: int, omega: Sequence[float], lam: float = HH_LAMBDA,
                         nb_rule=(1, 1), nq_rule=(1, 1), q0=0.0, scale=1.0,
                         name: str = "") -> Problem:
    """Chained Henon-Heiles problem (Eq. (18) with per-mode frequencies)."""
    omega = np.asarray(omega, np.float64).reshape(D)
    monos: List[tuple] = []
    for i in range(D):
        monos.append((0.5 * omega[i], [(i, 2)]))
    if lam != 0.0:
        for i in range(D - 1):
            monos.append((lam, [(i, 2), (i + 1, 1)]))
            monos.append((-lam / 3.0, [(i + 1, 3)]))
    coef, nfac, fmode, fpow = _poly(monos)
    full = lambda v, dt: np.full(D, v, dtype=dt)
    return Problem(D=D, L=L,
                   nb_A=full(nb_rule[0], np.int32), nb_B=full(nb_rule[1], np.int32),
                   nq_A=full(nq_rule[0], np.int32), nq_B=full(nq_rule[1], np.int32),
                   q0=full(q0, np.float64), scale=full(scale, np.float64),
                   omega=omega, coef=coef, nfac=nfac, fmode=fmode, fpow=fpow,
                   name=name or f"HH D={D} L={L}", meta={"lambda": lam})


def polynomial_problem(D: int, L: int, omega: Sequence[float], monos: Sequence[tuple],
                       nb_rule=(1, 1), nq_rule=(1, 1), q0=0.0, scale=1.0,
                       name: str = "") -> Problem:
    """General sparse-polynomial potential; monos = [(coef, [(mode, power), ...]), ...]."""
    coef, nfac, fmode, fpow = _poly(monos)
    full = lambda v, dt: np.full(D, v, dtype=dt)
    q0a = np.broadcast_to(np.asarray(q0, np.float64), (D,)).copy()
    sca = np.broadcast_to(np.asarray(scale, np.float64), (D,)).copy()
    return Problem(D=D, L=L,
                   nb_A=full(nb_rule[0], np.int32), nb_B=full(nb_rule[1], np.int32),
                   nq_A=full(nq_rule[0], np.int32), nq_B=full(nq_rule[1], np.int32),
                   q0=q0a, scale=sca, omega=np.asarray(omega, np.float64).reshape(D),
                   coef=coef, nfac=nfac, fmode=fmode, fpow=fpow, name=name or f"poly D={D} L={L}")


def draw_omega(D: int, seed: int, lo: float = 0.8, hi: float = 1.2) -> np.ndarray:
    """Per-mode frequencies omega_i ~ U[lo, hi] from a seeded PCG64 stream."""
    return np.random.Generator(np.random.PCG64(seed)).uniform(lo, hi, size=D)


def random_vectors(n: int, nvec: int, seed: int, normalise: bool = True) -> np.ndarray:
    """nvec seeded N(0,1) vectors of length n, column-major (shape (nvec, n)),
    each normalised to unit 2-norm when `normalise`."""
    g = np.random.Generator(np.random.PCG64(seed))
    x = g.standard_normal((nvec, n))
    if normalise and n > 0:
        x /= np.linalg.norm(x, axis=1, keepdims=True)
    return x


# ---- named workloads (sizes and distributions of the benchmark configurations) ----

def workload_C1(lam: float = HH_LAMBDA) -> Problem:
    """D=2 Henon-Heiles, omega=1, nb=nq=l+1, L=6 (FP64)."""
    return chained_henon_heiles(2, 6, [1.0, 1.0], lam, (1, 1), (1, 1), name="HH D=2 L=6 nb=nq=l+1")


def workload_C2(seed: int = 2, lam: float = HH_LAMBDA) -> Problem:
    """D=6 chained Henon-Heiles, omega_i ~ U[0.8,1.2], nb=nq=l+1, L=8."""
    return chained_henon_heiles(6, 8, draw_omega(6, seed), lam, (1, 1), (1, 1),
                                name="HH D=6 L=8 nb=nq=l+1")


def workload_C3(seed: int = 3, lam: float = HH_LAMBDA, L: int = 10, D: int = 12) -> Problem:
    """D=12 chained Henon-Heiles, omega_i ~ U[0.8,1.2], nb=l+1, nq=l+2, L=10."""
    return chained_henon_heiles(D, L, draw_omega(D, seed), lam, (1, 1), (2, 1),
                                name=f"HH D={D} L={L} nb=l+1 nq=l+2")


def coherent_factors(q0: Sequence[float], kw: int) -> np.ndarray:
    """1D Hermite-function coefficients c_n = exp(-a^2/2) a^n / sqrt(n!), a = q0/sqrt(2),
    n < kw, of a unit Gaussian displaced to q0 in each mode (a coherent state),
    shape (D, kw).  The product state over the compact basis is built by the
    library (sg_product_state) or the oracle's compact enumeration."""
    q0 = np.asarray(q0, np.float64)
    a = q0 / np.sqrt(2.0)
    out = np.empty((len(q0), kw))
    for i, ai in enumerate(a):
        c = np.empty(kw)
        c[0] = np.exp(-0.5 * ai * ai)
        for k in range(1, kw):
            c[k] = c[k - 1] * ai / np.sqrt(k)
        out[i] = c
    return out


def workload_C4(n: int = 256, seed: int = 4, Ds=(4, 6, 8, 10, 12), Ls=(6, 7, 8, 9, 10),
                lam: float = HH_LAMBDA):
    """Batch of n independent wavepacket problems: D uniform in Ds, L uniform in
    Ls, chained Henon-Heiles with omega_i ~ U[0.8,1.2], nb = nq = l+1, and a
    Gaussian wavepacket centred at q0_i ~ U[0,2] in every mode.
    Returns a list of (Problem, q0) pairs."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for j in range(n):
        D = int(g.choice(Ds))
        L = int(g.choice(Ls))
        om = g.uniform(0.8, 1.2, size=D)
        q0 = g.uniform(0.0, 2.0, size=D)
        out.append((chained_henon_heiles(D, L, om, lam, (1, 1), (1, 1),
                                         name=f"HH D={D} L={L} nb=nq=l+1 (batch item {j})"), q0))
    return out


def workload_C5(n: int, seed: int = 5, Ds=tuple(range(6, 21)), Ls=(4, 5, 6, 7, 8), steps=(20, 500),
                lam: float = HH_LAMBDA):
    """Stream of n propagation requests: D uniform in Ds, L uniform in Ls,
    chained Henon-Heiles with omega_i ~ U[0.8,1.2], nb = nq = l+1, a Gaussian
    wavepacket displaced by 2.0 in mode 0, steps uniform in [steps[0], steps[1]]
    (order 64, dt 0.1).  Returns a list of (Problem, q0, nsteps)."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for j in range(n):
        D = int(g.choice(Ds))
        L = int(g.choice(Ls))
        om = g.uniform(0.8, 1.2, size=D)
        nsteps = int(g.integers(steps[0], steps[1] + 1))
        q0 = np.zeros(D)
        q0[0] = 2.0
        out.append((chained_henon_heiles(D, L, om, lam, (1, 1), (1, 1),
                                         name=f"HH D={D} L={L} nb=nq=l+1 (request {j})"), q0, nsteps))
    return out
