"""CPU oracle for the pCGMG solve (Luu & Banh, arXiv 2301.07457).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the tests, the smoke check and the bench's
CPU-baseline leg use it.  It shares no code with the CUDA library (no kernels,
headers, constants or helpers) and never imports it.

It is plain, slow and FP64 throughout (numpy + scipy.sparse as library
primitives):
  * fem          -- Eq. 5 (multi-material SIMP), Eqs. 7-9 (Q4 plane-stress
                    element stiffness by 2x2 Gauss quadrature), assembly of K,
                    clamped edges, the element-by-element product K v, and the
                    direct solve u = K_ff^-1 f_f that defines the answer.
  * cholesky     -- Alg. 3 (dense Cholesky) with forward/back substitution.
  * multigrid    -- bilinear prolongation P and R = P^T (Sec. 2.1), Galerkin
                    and rediscretised coarse operators, damped Jacobi (Sec. 2.3),
                    the gamma-cycle of Alg. 1 (V- and W-cycle).
  * pcg          -- Alg. 2 (preconditioned conjugate gradient).
  * sensitivity  -- compliance C = f.u (Eq. 6) and the self-adjoint
                    sensitivity dC/dx_{e,i} = -p x^{p-1} E_i u_e^T KE u_e.
  * precision    -- round-to-nearest-even to bfloat16, for the mixed path.
  * solver       -- the whole pCGMG solve wired from the pieces above.
  * poisson      -- the scalar Poisson problem of Sec. 5.1 (Q4 Laplacian,
                    u = 0 on the boundary) on the same Alg. 1 / Alg. 2 pieces.

Every function names the passage of the paper it follows.  Readings of the
paper where it is silent or garbled are listed in the project's design notes;
the ones that change arithmetic are repeated in the docstrings here.
"""

from . import cholesky, fem, multigrid, pcg, poisson, precision, sensitivity, solver  # noqa: F401
