"""CPU oracle of the Smolyak operator action -- TEST INFRASTRUCTURE ONLY.

Three independent FP64 routes to y = H_S x (arXiv 2111.13655, Sec. 2-3):
  oracle.py     Eq. (16) term by term in plain C (via ctypes): every term
                through its full direct-product grid (Eqs. (14)-(15));
  galerkin.py   the masked-Galerkin closed form, valid where the quadrature of
                every term is exact;
  bruteforce.py dense Kronecker matrices for tiny problems.
Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this package; the CUDA library never does.
"""
