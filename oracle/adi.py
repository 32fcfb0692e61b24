"""Algorithm 1 (ADI) with the shift choice of Section 3, on the CPU with
banded solves (oracle package: test infrastructure and the timed CPU
baseline of the same algorithm only; the oracle proper solves every mode
directly, see ``sylvester``).

For the per-mode equation A Y B^T + C Y D^T = E of ``sylvester.ModeSystem``
(Section 3, eq. HelmholtzMatEqn), in the order of the paragraph that follows
Algorithm 1:

1. spectral intervals: [a, b] holds the eigenvalues of C^-1 A and [c, d] those
   of -D B^-1; here from the eigenvalues of the dense pencils of the operators
   (radial: mu of (-L_r, C); vertical: nu of (-D2, B)), widened by 5 %
   outward: [a, b] = [s + ka 0.95 mu_min, s + ka 1.05 mu_max] and
   [c, d] = [-ka 1.05 nu_max, -ka 0.95 nu_min] (s = 1, ka = kappa alpha for a
   heat step; s = 0, ka = 1 for Poisson);
2. gamma = |c - a||d - b| / (|c - b||d - a|), alpha = -1 + 2 gamma +
   2 sqrt(gamma^2 - gamma), k = sqrt(1 - 1/alpha^2), the complete elliptic
   integral K(k) and dn from scipy.special, and the Moebius map T with
   T(-alpha) = a, T(-1) = b, T(1) = c, T(alpha) = d;
3. J = ceil(log(16 gamma) log(4 / eps) / pi^2) (the text says only
   O(log mn); this J makes the Zolotarev bound 4 rho^(-2J) of the cited
   theorem at most eps);
4. shifts dn_j = dn((2j + 1) K / (2J), k): q_j = T(-alpha dn_j) in [a, b] and
   p_j = T(alpha dn_j) in [c, d];
5. from X_0 = 0, J iterations of the two half-steps, with the signs read so
   that the solution of the equation is the fixed point:
       (A - p_j C) X_{j+1/2} B^T = E - C X_j (D + p_j B)^T
       C X_{j+1} (D + q_j B)^T   = E - (A - q_j C) X_{j+1/2} B^T
   each half-step two banded solves (scipy.linalg.solve_banded), one on each
   side.  On eigenvectors the error is multiplied per iteration by
   (lam - q_j)(mu - p_j) / ((lam - p_j)(mu - q_j)), lam in [a, b],
   mu in [c, d]: the shift that enters the radial solve lies in the vertical
   spectrum and vice versa.  (As printed, the half-steps have the solution
   of the equation with -E as their fixed point, and the shift in [a, b]
   enters the radial solve, where the factor above needs one in [c, d].)
"""
import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.special as ss

from .sylvester import ModeSystem
from .transforms import slice_wavenumber

PAD = 0.05


def spectral_intervals(ms, kind, kappa_alpha=None):
    """(a, b, c, d) of step 1 for one ModeSystem (see the module docstring)."""
    mu = np.real(sla.eigvals(ms.dA, ms.C))          # -L_r against C: positive
    nu = np.real(sla.eigvals(ms.dD, ms.B))          # -D2 against B: positive
    s, ka = (0.0, 1.0) if kind == 'poisson' else (1.0, float(kappa_alpha))
    a = s + ka * (1 - PAD) * mu.min()
    b = s + ka * (1 + PAD) * mu.max()
    c = -ka * (1 + PAD) * nu.max()
    d = -ka * (1 - PAD) * nu.min()
    return a, b, c, d


def mobius(z, w):
    """The Moebius map T(x) = (P x + Q) / (R x + S) with T(z_i) = w_i for three
    distinct points (the null vector of the three linear conditions)."""
    Mx = np.array([[zi, 1.0, -wi * zi, -wi] for zi, wi in zip(z, w)])
    P, Q, R, S = sla.null_space(Mx)[:, 0]
    return lambda x: (P * np.asarray(x) + Q) / (R * np.asarray(x) + S)


def zolotarev_shifts(a, b, c, d, tol):
    """Steps 2 to 4: (J, p shifts in [c, d], q shifts in [a, b], gamma, alpha, T)."""
    gamma = abs(c - a) * abs(d - b) / (abs(c - b) * abs(d - a))
    alpha = -1.0 + 2.0 * gamma + 2.0 * math.sqrt(gamma * gamma - gamma)
    J = max(1, math.ceil(math.log(16.0 * gamma) * math.log(4.0 / tol) / math.pi ** 2))
    m1 = 1.0 / alpha ** 2                           # 1 - k^2
    K = ss.ellipkm1(m1)
    T = mobius((-alpha, -1.0, 1.0), (a, b, c))
    dn = np.array([ss.ellipj((2 * j + 1) * K / (2 * J), 1.0 - m1)[2] for j in range(J)])
    return J, T(alpha * dn), T(-alpha * dn), gamma, alpha, T


def _banded(M):
    """(l, u) and the solve_banded storage of a dense banded matrix."""
    nz = np.nonzero(M)
    off = nz[1] - nz[0]
    lo, up = max(0, -off.min()), max(0, off.max())
    n = M.shape[0]
    ab = np.zeros((lo + up + 1, n))
    for o in range(-lo, up + 1):
        dg = np.diagonal(M, o)
        if o >= 0:
            ab[up - o, o:] = dg
        else:
            ab[up - o, :n + o] = dg
    return (lo, up), ab


def _solve(M, R):
    lu, ab = _banded(M)
    return sla.solve_banded(lu, ab, R)


def adi_solve(ms, E, p, q):
    """Step 5: J = len(p) iterations from X_0 = 0 of the half-steps above."""
    A, B, C, D = (sp.csr_matrix(x) for x in (ms.A, ms.B, ms.C, ms.D))
    X = np.zeros_like(E)
    for pj, qj in zip(p, q):
        # (A - p C) X_half B^T = E - C X (D + p B)^T
        R1 = E - C @ ((D + pj * B) @ X.T).T
        W = _solve(ms.A - pj * ms.C, R1)            # W = X_half B^T
        X_half = _solve(ms.B, W.T).T
        # C X_new (D + q B)^T = E - (A - q C) X_half B^T
        R2 = E - (A - qj * C) @ (B @ X_half.T).T
        V = _solve(ms.C, R2)                        # V = X_new (D + q B)^T
        X = _solve(ms.D + qj * ms.B, V.T).T
    return X


class _adi_systems(dict):
    """ModeSystem and shifts per distinct |k|, built on first use."""

    def __init__(self, m, n, kind, kappa_alpha, tol):
        super().__init__()
        self.args = (m, n, kind, kappa_alpha, tol)

    def __missing__(self, k):
        m, n, kind, ka, tol = self.args
        ms = ModeSystem(m, n, k, kind, ka)
        J, p, q, _, _, _ = zolotarev_shifts(*spectral_intervals(ms, kind, ka), tol)
        self[k] = (ms, p, q)
        return self[k]


def poisson(F, tol, slices=None):
    """-lap u = f (zero Dirichlet data) with every mode solved by ADI."""
    p, m, n = F.shape
    sys_ = _adi_systems(m, n, 'poisson', None, tol)
    U = np.zeros_like(F)
    for s in (range(p) if slices is None else slices):
        ms, ps, qs = sys_[slice_wavenumber(s, p)]
        U[s] = ms.expand(adi_solve(ms, ms.rhs(F[s]), ps, qs))
    return U


def heat_steps(X0, g, alpha, dt, nsteps, tol, slices=None):
    """BDF1 steps (constant forcing g, level n for step n -> n+1) with every
    mode solved by ADI."""
    p, m, n = X0.shape
    sys_ = _adi_systems(m, n, 'heat', dt * alpha, tol)
    X = np.array(X0, dtype=np.float64, copy=True)
    todo = list(range(p) if slices is None else slices)
    for _ in range(nsteps):
        Xn = np.zeros_like(X)
        for s in todo:
            ms, ps, qs = sys_[slice_wavenumber(s, p)]
            Xn[s] = ms.expand(adi_solve(ms, ms.rhs(X[s] + dt * g[s]), ps, qs))
        X = Xn
    return X
