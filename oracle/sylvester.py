"""Per-Fourier-mode matrix equation and its direct solution (oracle; test infrastructure only).

Section 3, eq. HelmholtzMatEqn: for each wavenumber k the BDF step is the
generalised Sylvester equation

    (R_2 - kappa alpha (R C12 D1 + R^2 D2 - k^2 C02)) X C02^T
        - kappa alpha R_2 X D2^T = R_2 (delta X + kappa g) C02^T ,

and the Poisson problem -lap u = f (Section 4, the Poisson solves, and the
remark that the same machinery solves it) is the same equation with the identity
term removed and the sign of the Laplacian flipped:

    -(R C12 D1 + R^2 D2 - k^2 C02) U C02^T - R_2 U D2^T = R_2 F C02^T .

Reading of the unstated boundary conditions: homogeneous Dirichlet data at
r = +-1 and z = +-1, imposed by X = S_r Y S_z^T (S = ``dirichlet_basis``)
and by keeping the first m-2 rows / n-2 columns of the C^(2) equations.
Per mode this gives   A Y B^T + C Y D^T = E   with (m-2) x (m-2) matrices
A, C and (n-2) x (n-2) matrices B, D.

Algorithm 1 (ADI) approximates the solution of exactly this equation; the
oracle solves it directly instead:
* ``solve_kron``  -- brute force: dense LU of (B kron A + D kron C).
* ``BartelsStewart`` -- generalised Bartels-Stewart through the QZ
                     decomposition of the pencils (A, C) and (B, D).
"""
import numpy as np
import scipy.linalg as sla

from . import operators as ops


class ModeSystem:
    """A, B, C, D of one wavenumber k (both radial parities, full size)."""

    def __init__(self, m, n, k, kind, kappa_alpha=None):
        Pr, Pz = ops.tau_rows(m), ops.tau_rows(n)
        Sr, Sz = ops.dirichlet_basis(m), ops.dirichlet_basis(n)
        R2r = ops.r2_C2(m)
        Lk = ops.radial_laplacian_r2(m, k)
        self.C = Pr @ R2r @ Sr
        self.B = Pz @ ops.conv_T_to_C2(n) @ Sz
        D2z = Pz @ ops.diff2_T_to_C2(n) @ Sz
        Lr = Pr @ Lk @ Sr
        if kind == 'poisson':
            self.A = -Lr
            self.D = -D2z
        elif kind == 'heat':
            ka = float(kappa_alpha)
            self.A = self.C - ka * Lr
            self.D = -ka * D2z
        else:
            raise ValueError(kind)
        # derivatives w.r.t. kappa*alpha (used by the adjoint)
        self.dA = -Lr
        self.dD = -D2z
        self.m, self.n, self.k = m, n, k
        # the equation's left operator on a full T-coefficient block (for lifting)
        Lk_full, C02z, D2z_full = Lk, ops.conv_T_to_C2(n), ops.diff2_T_to_C2(n)
        if kind == 'poisson':
            self._full = [(-Pr @ Lk_full, Pz @ C02z), (-Pr @ R2r, Pz @ D2z_full)]
        else:
            ka = float(kappa_alpha)
            self._full = [(Pr @ (R2r - ka * Lk_full), Pz @ C02z), (-ka * Pr @ R2r, Pz @ D2z_full)]
        # its derivative w.r.t. kappa*alpha (heat; used by the adjoint with lifting)
        self._dfull = [(-Pr @ Lk_full, Pz @ C02z), (-Pr @ R2r, Pz @ D2z_full)]
        # right-hand-side map E = P_r R_2 Z C02^T P_z^T, and X = S_r Y S_z^T
        self.rhs_left = Pr @ R2r
        self.rhs_right = (Pz @ ops.conv_T_to_C2(n)).T
        self.Sr, self.Sz = Sr, Sz

    def rhs(self, Z):
        """E = trunc(R_2 Z C02^T) for a T-coefficient block Z (m x n)."""
        return self.rhs_left @ Z @ self.rhs_right

    def rhs_T(self, Lam):
        """Transpose of ``rhs`` (Frobenius inner product)."""
        return self.rhs_left.T @ Lam @ self.rhs_right.T

    def expand(self, Y):
        """X = S_r Y S_z^T."""
        return self.Sr @ Y @ self.Sz.T

    def expand_T(self, X):
        return self.Sr.T @ X @ self.Sz

    def full_apply(self, U):
        """Left side of the equation on a full T-coefficient block U (m x n)."""
        return sum(Am @ U @ Bm.T for Am, Bm in self._full)

    def full_apply_dka(self, U):
        """Derivative of ``full_apply(U)`` w.r.t. kappa*alpha (heat)."""
        return sum(Am @ U @ Bm.T for Am, Bm in self._dfull)

    def apply(self, Y):
        """Left side of the equation: A Y B^T + C Y D^T."""
        return self.A @ Y @ self.B.T + self.C @ Y @ self.D.T


def solve_kron(A, B, C, D, E):
    """Brute force: vec(A Y B^T + C Y D^T) = (B kron A + D kron C) vec(Y),
    column-major vec, solved by dense LU.  For tiny sizes only."""
    K = np.kron(B, A) + np.kron(D, C)
    y = np.linalg.solve(K, E.reshape(-1, order='F'))
    return y.reshape(E.shape, order='F')


class BartelsStewart:
    """Direct solver of A Y B^T + C Y D^T = E for fixed (A, B, C, D).

    Generalised Bartels-Stewart (the QZ form of Gardiner, Laub, Amato and
    Moler): complex QZ of the two pencils, A = Q1 S1 Z1^H, C = Q1 T1 Z1^H and
    B = Q2 S2 Z2^H, D = Q2 T2 Z2^H with S, T upper triangular.  With
    W = Z1^H Y conj(Z2) the equation becomes S1 W S2^T + T1 W T2^T =
    Q1^H E conj(Q2), whose columns are found from the last to the first:
        (S2[j,j] S1 + T2[j,j] T1) w_j
            = e_j - S1 sum_{l>j} S2[j,l] w_l - T1 sum_{l>j} T2[j,l] w_l .
    Then Y = Z1 W Z2^T.  No matrix is inverted explicitly, so the solve is
    backward stable; the QZ forms are computed once per matrix set."""

    def __init__(self, A, B, C, D):
        self.fwd = _QZSylv(A, B, C, D)
        self._args = (A, B, C, D)
        self.bwd = None

    def solve(self, E):
        return self.fwd.solve(E)

    def solve_T(self, M):
        """Solve the transposed equation A^T L B + C^T L D = M, i.e. the same
        form with every matrix transposed."""
        if self.bwd is None:
            A, B, C, D = self._args
            self.bwd = _QZSylv(A.T, B.T, C.T, D.T)
        return self.bwd.solve(M)


class _QZSylv:
    def __init__(self, A, B, C, D):
        self.S1, self.T1, self.Q1, self.Z1 = sla.qz(A, C, output='complex')
        self.S2, self.T2, self.Q2, self.Z2 = sla.qz(B, D, output='complex')

    def solve(self, E):
        S1, T1, S2, T2 = self.S1, self.T1, self.S2, self.T2
        Et = self.Q1.conj().T @ E @ self.Q2.conj()
        m, n = Et.shape
        W = np.zeros((m, n), dtype=np.complex128)
        SW = np.zeros((m, n), dtype=np.complex128)      # S1 @ W, columns filled as solved
        TW = np.zeros((m, n), dtype=np.complex128)      # T1 @ W
        for j in range(n - 1, -1, -1):
            rhs = Et[:, j] - SW[:, j + 1:] @ S2[j, j + 1:] - TW[:, j + 1:] @ T2[j, j + 1:]
            M = S2[j, j] * S1 + T2[j, j] * T1
            W[:, j] = sla.solve_triangular(M, rhs, lower=False)
            SW[:, j] = S1 @ W[:, j]
            TW[:, j] = T1 @ W[:, j]
        return (self.Z1 @ W @ self.Z2.T).real


def bordered_solve(m, n, k, kind, kappa_alpha, rhs_coeffs, wall):
    """Brute force with boundary data, one slice: the tau equations of the
    mode (the first m-2 x n-2 C^(2) rows of eq. HelmholtzMatEqn or its
    Poisson form, acting on the full T-coefficient block U) bordered by the
    Dirichlet rows  sum_j U[j,:] T_j(+-1) = traces of the data at r = +-1 and
    sum_k U[:,k] T_k(+-1) = traces at z = +-1.  `wall` is the T-coefficient
    block of any function with the required boundary traces (its interior
    does not matter); the bordered system is assembled densely and solved by
    least squares (it is consistent; the corner rows are redundant).

    rhs_coeffs: Z with right side trunc(R_2 Z C02^T)."""
    Pr, Pz = ops.tau_rows(m), ops.tau_rows(n)
    R2r, C02r, C02z = ops.r2_C2(m), ops.conv_T_to_C2(m), ops.conv_T_to_C2(n)
    Lk = ops.radial_laplacian_r2(m, k)
    D2z = ops.diff2_T_to_C2(n)
    if kind == 'poisson':
        left = [(-Pr @ Lk, Pz @ C02z), (-Pr @ R2r, Pz @ D2z)]
    else:
        ka = float(kappa_alpha)
        left = [(Pr @ (R2r - ka * Lk), Pz @ C02z), (-ka * Pr @ R2r, Pz @ D2z)]
    # vec(A U B^T) = (B kron A) vec(U), column-major
    K = sum(np.kron(Bm, Am) for Am, Bm in left)
    rhs = (Pr @ R2r @ rhs_coeffs @ (Pz @ C02z).T).reshape(-1, order='F')
    ends_r = np.array([[(-1.0) ** j for j in range(m)], [1.0] * m])   # T_j(-1), T_j(1)
    ends_z = np.array([[(-1.0) ** j for j in range(n)], [1.0] * n])
    rows, vals = [], []
    for e in range(2):       # r = -1, +1: sum_j U[j, kk] T_j(end) for every kk
        for kk in range(n):
            Ei = np.zeros((m, n)); Ei[:, kk] = ends_r[e]
            rows.append(Ei.reshape(-1, order='F')); vals.append(ends_r[e] @ wall[:, kk])
    for e in range(2):       # z = -1, +1
        for j in range(m):
            Ei = np.zeros((m, n)); Ei[j, :] = ends_z[e]
            rows.append(Ei.reshape(-1, order='F')); vals.append(wall[j, :] @ ends_z[e])
    Kb = np.vstack([K, np.array(rows)])
    b = np.concatenate([rhs, np.array(vals)])
    u = np.linalg.lstsq(Kb, b, rcond=None)[0]
    return u.reshape((m, n), order='F')
