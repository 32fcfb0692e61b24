"""Ultraspherical operators of Section 3 (oracle; test infrastructure only).

All matrices are dense float64, square of the requested size, and act on
coefficient column vectors (index = polynomial degree).  They are built from
the classical relations between the Chebyshev T, U = C^(1) and C^(2) families
in the Abramowitz-Stegun normalisation named in Section 2, not from the
printed matrices; the tests compare them with the printed entries.

Readings (also in the design notes):
* C01 is printed as a zero-diagonal tridiagonal with 1/2 off the diagonal,
  which is not the T -> U conversion the text says it is.  ``conv_T_to_U``
  builds the conversion that the text names: T_0 = U_0, T_1 = U_1 / 2,
  T_j = (U_j - U_{j-2}) / 2.
* The printed D1 is the T -> U derivative (d/dx T_j = j U_{j-1}); the printed
  D2 is the T -> C^(2) second derivative (d^2/dx^2 T_j = 2 j C^(2)_{j-2}), the
  relation Section 2 states with a garbled argument ("T_K(x^2)").
"""
import numpy as np


def conv_T_to_U(m):
    """C01 of Section 3 (operator list): T coefficients -> U coefficients."""
    M = np.zeros((m, m))
    for j in range(m):
        if j == 0:
            M[0, 0] = 1.0
        else:
            M[j, j] = 0.5
            if j >= 2:
                M[j - 2, j] = -0.5
    return M


def conv_U_to_C2(m):
    """C12 of Section 3: U = C^(1) coefficients -> C^(2) coefficients.

    From C^(1)_j = (C^(2)_j - C^(2)_{j-2}) / (j + 1)."""
    M = np.zeros((m, m))
    for j in range(m):
        M[j, j] = 1.0 / (j + 1.0)
        if j >= 2:
            M[j - 2, j] = -1.0 / (j + 1.0)
    return M


def conv_T_to_C2(m):
    """C02 = C12 C01 of Section 3."""
    return conv_U_to_C2(m) @ conv_T_to_U(m)


def mult_r_C2(m):
    """R of Section 3: multiplication by r of a C^(2) coefficient vector.

    From x C^(2)_j = ((j + 1) C^(2)_{j+1} + (j + 3) C^(2)_{j-1}) / (2 (j + 2))."""
    M = np.zeros((m, m))
    for j in range(m):
        if j + 1 < m:
            M[j + 1, j] = (j + 1.0) / (2.0 * j + 4.0)
        if j >= 1:
            M[j - 1, j] = (j + 3.0) / (2.0 * j + 4.0)
    return M


def r2_C2(m):
    """R_2 = R^2 C02 of Section 3: T coefficients -> C^(2) coefficients of r^2 f."""
    R = mult_r_C2(m)
    return R @ R @ conv_T_to_C2(m)


def diff1_T_to_U(m):
    """D1 of Section 3: d/dx T_j = j U_{j-1}."""
    M = np.zeros((m, m))
    for j in range(1, m):
        M[j - 1, j] = float(j)
    return M


def diff2_T_to_C2(m):
    """D2 of Section 3: d^2/dx^2 T_j = 2 j C^(2)_{j-2}."""
    M = np.zeros((m, m))
    for j in range(2, m):
        M[j - 2, j] = 2.0 * j
    return M


def radial_laplacian_r2(m, k):
    """r^2 (d_r^2 + r^-1 d_r - k^2 r^-2) in the C^(2) output basis.

    The left operator of eq. Helmholtz without its identity and z terms:
    R C12 D1 + R^2 D2 - k^2 C02 (eq. HelmholtzMatEqn)."""
    R = mult_r_C2(m)
    return R @ conv_U_to_C2(m) @ diff1_T_to_U(m) + R @ R @ diff2_T_to_C2(m) \
        - float(k) ** 2 * conv_T_to_C2(m)


def dirichlet_basis(m):
    """Recombination S (m x (m-2)): column j holds phi_j = T_{j+2} - T_j.

    Reading of the unstated boundary conditions: phi_j(+-1) = 0, so
    X = S Y meets homogeneous Dirichlet data at both ends of the doubled
    radial interval (r = -1 is the physical wall at theta + pi) and of z."""
    S = np.zeros((m, m - 2))
    for j in range(m - 2):
        S[j, j] = -1.0
        S[j + 2, j] = 1.0
    return S


def tau_rows(m):
    """P (m-2 x m): keep the first m-2 equations of a C^(2) expansion (tau)."""
    P = np.zeros((m - 2, m))
    P[:, : m - 2] = np.eye(m - 2)
    return P
