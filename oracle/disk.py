"""Horizontal (disk) Poisson solve of the poloidal-toroidal decomposition
(oracle; test infrastructure only).

Section 4, eq. ptpoisson: the toroidal and poloidal potentials follow from
-Delta_h u = f, Delta_h = lap - d_z^2 = r^-1 d_r + d_r^2 + r^-2 d_theta^2, the
Laplacian without its vertical term.  The paper solves it by diagonalising in
theta and z; here z is a pure parameter (no z derivative, no z boundary
condition), so every z-coefficient column of every half-complex slice is an
independent radial problem with u = 0 at r = -1 and r = +1 (the wall of the
doubled grid; reading of the unstated boundary conditions).  Discretisation:
the r^2-multiplied radial operator of Section 3 (eq. HelmholtzMatEqn without
its z terms) in the same ultraspherical tau form,

    trunc(-L_k S_r) y = trunc(R_2 f),   u = S_r y,

L_k = R C12 D1 + R^2 D2 - k^2 C02, S_r the Dirichlet recombination
phi_j = T_{j+2} - T_j, trunc = the first m - 2 C^(2) rows.
"""
import numpy as np

from . import operators as ops
from .transforms import slice_wavenumber


def horizontal_poisson(F, slices=None):
    """Coefficients u of -Delta_h u = f for half-complex coefficients F
    ([p][m][n]); dense solve of the (m-2) x (m-2) radial tau system per
    wavenumber."""
    F = np.asarray(F, dtype=np.float64)
    p, m, n = F.shape
    Pr, Sr, R2 = ops.tau_rows(m), ops.dirichlet_basis(m), ops.r2_C2(m)
    U = np.zeros_like(F)
    cache = {}
    for s in (range(p) if slices is None else slices):
        k = slice_wavenumber(s, p)
        if k not in cache:
            cache[k] = -Pr @ ops.radial_laplacian_r2(m, k) @ Sr
        Y = np.linalg.solve(cache[k], Pr @ R2 @ F[s])
        U[s] = Sr @ Y
    return U
