"""FP64 CPU oracle for the real-space RPA correlation-energy method (arXiv 2504.01816).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import, call or link anything in this package.
The product (the CUDA library and its Python binding) never does.

Parity status of each function (what pins it, see tests/test_oracle_pins.py):
  fd_weights            textbook 12th-order weights (golden file) and polynomial exactness
  apply_h               dense Hamiltonian assembled independently; polynomial exactness
  Coulomb.apply         dense inverse of -L_h; nu^1/2 nu^1/2 = nu; point-charge limit
  cocg                  dense complex solve
  Oracle.chi0           brute-force sum over states from a full dense eigendecomposition
                        (Eq. 2); invariants chi0 1 = 0, symmetry, negative semi-definite
  Oracle.chi0(galerkin) equal to the projected form (cancellation argument)
  frequency_quadrature  closed-form integrals of rational functions on [0, inf)
  rpa_ec                dense eigenvalues of nu^1/2 chi0 nu^1/2 at full rank; adaptive
                        quadrature of the dense integrand; convergence in N_omega
  rpa_ec_gradient       central finite differences of a dense sum-over-states E_c built
                        from the unoccupied eigenpairs of the projected Hamiltonian
  periodic grids        the stencil's closed-form symbol on Fourier modes, plane waves, dense
                        pseudo-inverses, sum over states (tests/test_oracle_pins_periodic.py)
  laplacian_preconditioner  dense inverse of -1/2 L_h + shift
  pcocg                 dense complex solve; with a multiple of the identity as M it is COCG
                        (same iterates as cocg); fewer iterations than cocg at small omega
  block_cocg            one column is cocg (same iterates); dense complex solve; finite
                        termination in ceil(N / s) steps on an N-dimensional operator; block
                        orthogonality of the residuals and block A-conjugacy of the directions
                        (tests/test_oracle_pins_block.py)
  gauss_sq_trace        exactness for polynomials of degree <= 2 N_o - 1 (Gauss rule); order 1
                        is sum f(C_rr); order >= the dimension is Tr f(C) by dense eigenvalues
"""
from .rpa_oracle import *  # noqa: F401,F403
from .rpa_oracle import (Oracle, Grid, Coulomb, SolveStats, EcResult, fd_weights, apply_h, cocg,  # noqa: F401
                         frequency_quadrature, g_rpa, orthonormalize_cholesky, rpa_ec, num_threads,
                         set_threads, second_difference_1d, NotSPD, rpa_ec_gradient, gauss_sq_trace,
                         laplacian_preconditioner, pcocg, block_cocg, block_cocg_generic)
