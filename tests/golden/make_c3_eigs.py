"""Writes tests/golden/c3_eigs.txt: the 20 lowest eigenvalues of the Smolyak
Hamiltonian of the D=12 L=10 chained Henon-Heiles workload (nb = l+1,
nq = l+2, omega_i ~ U[0.8,1.2] with seed 3, lambda = 0.111803).

At nq = l+2 every quadrature of this cubic Hamiltonian is exact, so H_S is the
masked Galerkin matrix of oracle/galerkin.py (Eq. (16) collapsed by the
combination identity of Eq. (8)); its lowest eigenvalues come from scipy's
Lanczos (eigsh) in FP64.  Calls only oracle/ and the seeded input definitions.

    python tests/golden/make_c3_eigs.py
"""
import os
import sys
import time

import numpy as np
import scipy.sparse.linalg as sla

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import galerkin  # noqa: E402
from paper_2111_13655_gb300 import synth  # noqa: E402


def main():
    p = synth.workload_C3()
    t0 = time.time()
    H = galerkin.matrix(p)
    t1 = time.time()
    asym = abs(H - H.T).max()
    v0 = np.random.default_rng(2024).standard_normal(H.shape[0])
    w, V = sla.eigsh(H, k=20, which="SA", tol=1e-13, v0=v0, ncv=80, maxiter=20000)
    order = np.argsort(w)
    w, V = w[order], V[:, order]
    res = np.linalg.norm(H @ V - V * w, axis=0)
    t2 = time.time()
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c3_eigs.txt")
    with open(out, "w") as f:
        f.write("# 20 lowest eigenvalues of H_S, chained Henon-Heiles D=12 L=10, nb=l+1, nq=l+2,\n")
        f.write("# omega_i ~ U[0.8,1.2] (PCG64 seed 3), lambda=0.111803: masked Galerkin matrix\n")
        f.write(f"# (oracle/galerkin.py, N={H.shape[0]}, nnz={H.nnz}, max|H-H^T|={asym:.1e}),\n")
        f.write(f"# scipy eigsh (FP64); max residual norm {res.max():.2e}.  Written by make_c3_eigs.py.\n")
        for e in w:
            f.write(f"{e:.15e}\n")
    print(f"assembly {t1 - t0:.1f} s, eigsh {t2 - t1:.1f} s, max residual {res.max():.2e} -> {out}")


if __name__ == "__main__":
    main()
