"""Value <-> coefficient maps of the CCF interpolant (oracle; test infrastructure only).

Section 2, interpolant: f*(r, z, theta) = sum_{j,k,l} f^(j,k,l) T_j(r) T_k(z)
exp(i (l - floor(p/2)) theta), equal to f on the grid of Definition "grid".
The forward map is the DCT-I in r, the DCT-I in z and the DFT in theta
(Section 2, the three-stage transform); here each stage is its plain direct
sum, so the result is the interpolation coefficients with no fast algorithm.

Array layout (values and coefficients alike): [p][m][n] = [theta][r][z].

Half-complex coefficient storage used throughout the repository (real
fields only, p even): slice 0 holds c_0; slices 2w-1 and 2w hold Re c_w and
Im c_w for w = 1 .. p/2-1; slice p-1 holds c_{-p/2}, which is real on the
doubled grid.  Negative wavenumbers follow from c_{-w} = conj(c_w).
"""
import numpy as np
from numpy.polynomial import chebyshev as npcheb

from . import grid


def _cheb_forward_matrix(m):
    """DCT-I of Section 2 as a matrix: c_j = (2/(m-1)) w_j sum_a w_a f_a T_j(x_a),
    w = 1/2 at both ends, else 1 (discrete orthogonality of T_j at the
    Chebyshev extreme points)."""
    x = grid.cheb_points(m)
    V = npcheb.chebvander(x, m - 1)          # V[a, j] = T_j(x_a)
    w = np.ones(m)
    w[0] = w[-1] = 0.5
    return (2.0 / (m - 1)) * (w[:, None] * (V * w[:, None]).T)


def _cheb_inverse_matrix(m):
    """Evaluation of a T-series at the grid: f_a = sum_j c_j T_j(x_a)."""
    return npcheb.chebvander(grid.cheb_points(m), m - 1)


def vals2coeffs_complex(f):
    """Values [p][m][n] (real or complex) -> full complex coefficients
    C[l][j][k] on wavenumber w = l - floor(p/2) (Section 2 transform order:
    r, then z, then theta)."""
    p, m, n = f.shape
    Wr = _cheb_forward_matrix(m)
    Wz = _cheb_forward_matrix(n)
    g = np.einsum('ja,lab->ljb', Wr, f)          # DCT-I along r
    g = np.einsum('kb,ljb->ljk', Wz, g)          # DCT-I along z
    th = grid.theta_points(p)
    w = grid.wavenumbers(p)
    E = np.exp(-1j * np.outer(w, th)) / p        # c_w = (1/p) sum_l f_l e^{-i w theta_l}
    return np.einsum('wl,ljk->wjk', E, g)


def coeffs2vals_complex(C):
    """Full complex coefficients -> values of the interpolant on the grid."""
    p, m, n = C.shape
    Vr = _cheb_inverse_matrix(m)
    Vz = _cheb_inverse_matrix(n)
    th = grid.theta_points(p)
    w = grid.wavenumbers(p)
    E = np.exp(1j * np.outer(th, w))             # E[l, w] = e^{i w theta_l}
    g = np.einsum('lw,wjk->ljk', E, C)
    g = np.einsum('aj,ljk->lak', Vr, g)
    return np.einsum('bk,lak->lab', Vz, g)


def slice_wavenumber(s, p):
    """|wavenumber| carried by half-complex slice s."""
    if s == 0:
        return 0
    if s == p - 1:
        return p // 2
    return (s + 1) // 2


def complex_to_halfcomplex(C):
    """Full complex coefficients (index l, w = l - p/2) -> half-complex real slices."""
    p = C.shape[0]
    assert p % 2 == 0
    h = p // 2
    H = np.zeros(C.shape, dtype=np.float64)
    H[0] = C[h].real                              # w = 0
    for w in range(1, h):
        H[2 * w - 1] = C[h + w].real
        H[2 * w] = C[h + w].imag
    H[p - 1] = C[0].real                          # w = -p/2
    return H


def halfcomplex_to_complex(H):
    """Inverse of ``complex_to_halfcomplex`` (Hermitian completion)."""
    p = H.shape[0]
    h = p // 2
    C = np.zeros(H.shape, dtype=np.complex128)
    C[h] = H[0]
    for w in range(1, h):
        c = H[2 * w - 1] + 1j * H[2 * w]
        C[h + w] = c
        C[h - w] = np.conj(c)
    C[0] = H[p - 1]
    return C


def vals2coeffs(f):
    """Real values [p][m][n] -> half-complex coefficients [p][m][n]."""
    return complex_to_halfcomplex(vals2coeffs_complex(np.asarray(f, dtype=np.float64)))


def coeffs2vals(H):
    """Half-complex coefficients -> real values on the grid."""
    return coeffs2vals_complex(halfcomplex_to_complex(H)).real
