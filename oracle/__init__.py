"""Plain, slow FP64 CPU oracle for the Chebyshev-Chebyshev-Fourier cylinder solver
(Darrow, "A Quasi-Optimal Spectral Solver for the Heat and Poisson Equations in a
Closed Cylinder", arXiv 2206.04827).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import it.  The CUDA library never calls it,
and it shares no code with the CUDA library (no kernels, headers, tables or
helpers).  Every function cites the passage of the paper it restates.

What the oracle computes (all in float64, dense matrices, no blocking or fusion):

* ``grid``        -- the doubled CCF grid (Section 2, Definition "grid").
* ``transforms``  -- value <-> coefficient maps of the unique CCF interpolant
                     (Section 2, interpolant f*), written as direct sums.
* ``operators``   -- the ultraspherical conversion, multiplication and
                     differentiation matrices C01, C12, C02, R, R_2, D1, D2
                     (Section 3, operator list) built from the classical
                     three-term relations, plus the Dirichlet recombination.
* ``sylvester``   -- the per-Fourier-mode matrix equation (eq. HelmholtzMatEqn
                     and its Poisson analogue), solved directly: a dense
                     Kronecker solve (tiny sizes, brute force) and a
                     Bartels-Stewart solve (moderate sizes).  The ADI method of
                     Algorithm 1 converges to exactly this solution, so the
                     direct solve is the definition of record.
* ``heat``        -- Poisson driver, BDF1 time stepping (Section 3, BDF 1) and
                     the discrete adjoint of the stepping (chain rule through the
                     direct solves).

Readings of passages that are garbled or silent (each also listed in the
design notes of the repository):

* C01 as printed is not the T->U conversion it is described as; the oracle
  builds the T->U conversion that the text names.
* Eq. HelmholtzMatEqn writes ell^2 for the angular term; the oracle uses k^2
  with k = ell - floor(p/2), the wavenumber of the basis (Section 2, CCF
  polynomial).
* Boundary conditions are not stated for the heat or Poisson problem: the
  oracle imposes homogeneous Dirichlet data at r = +-1 and z = +-1 by
  recombination (phi_j = T_{j+2} - T_j) and keeps the first m-2 (n-2)
  rows of each C^(2) equation (tau method).
* BDF order of the experiments is not stated: BDF1 (kappa = h), with the
  forcing of step n -> n+1 taken at time level n (the extrapolation
  g(t+h) ~ g(t) stated beside eq. HelmholtzMatEqn).

Parity is pinned for every function: see ``tests/test_oracle_*.py``.
"""
