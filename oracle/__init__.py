"""FP64 CPU oracle for the compact Runge--Kutta discontinuous Galerkin (cRKDG)
method of Chen, Sun and Xing, "The Runge--Kutta discontinuous Galerkin method
with compact stencils for hyperbolic conservation laws" (arXiv 2307.06471).

THIS PACKAGE IS TEST INFRASTRUCTURE.  It is a plain, slow, obviously correct
restatement of the paper's scheme in numpy float64, written to be checked
against the paper by eye.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  The CUDA library never calls
it, and it never calls the CUDA library: the two share no code, tables or
constants.

Layout of a 1D state:  u[x, v, m]       (cell, variable, Legendre mode)
Layout of a 2D state:  u[y, x, v, m]    (row, column, variable, mode)

Modules
  basis      Legendre bases, Gauss rules, 2D mode sets (Sec. 2.1 space V_h)
  physics    fluxes, wave speeds, LF/LLF numerical flux, Euler eigenvectors
  dg1d       1D operators (DG operator, eq. (2.3); local operator, eq. (2.7))
             and the RKDG (eq. (2.6)), cRKDG (eq. (2.8)) and Shu--Osher
             variants (Sec. 3.2.1, eqs. (3.1)-(3.3))
  dg2d       the same on 2D Cartesian meshes, with boundary conditions
  limiter    TVB-minmod limiter in characteristic fields (Sec. 4.2; reading stated)
  problems   exact solutions and initial data of the paper's tests (Sec. 4)
  norms      L1 / L2 / Linf error norms by Gauss quadrature
  vonneumann maximum stable CFL numbers by eigenvalues of the step matrix (Table 1.1)
  mlp        the troubled-cell indicator MLP: forward, backward, Adam (FP64)

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` except the TVB-minmod limiter, whose details the
paper cites but does not print ("parity unpinned" against the paper; it is
pinned by invariants only), and the MLP feature recipe, which the paper does
not contain at all (pinned by finite differences only).
"""
