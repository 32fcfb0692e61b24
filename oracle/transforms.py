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

from . import grid


def _cos_pi_ratio(r, d):
    """cos(pi r / d) for integer arrays r, d > 0: r is reduced exactly modulo
    2d in integers and folded to an angle in [0, pi/2] before the cosine, so
    large degrees or wavenumbers add no rounding of their own."""
    r = np.mod(np.asarray(r, dtype=np.int64), 2 * d)
    r = np.where(r > d, 2 * d - r, r)                 # cos is even about pi
    sign = np.where(2 * r > d, -1.0, 1.0)             # cos(pi - t) = -cos(t)
    r = np.where(2 * r > d, d - r, r)
    return sign * np.cos(np.pi * r / d)


def _cheb_at_grid(m):
    """T[a, j] = T_j(x_a) on the grid of Definition "grid", from the defining
    identity T_j(cos t) = cos(j t) with x_a = cos((m-1-a) pi / (m-1))."""
    N = m - 1
    a = np.arange(m, dtype=np.int64)[:, None]
    j = np.arange(m, dtype=np.int64)[None, :]
    return _cos_pi_ratio(j * (N - a), N)


def _fourier_at_grid(p, sign):
    """E[w, l] = exp(sign i w theta_l) for w = l' - p/2 (Section 2, CCF
    polynomial) and theta_l = (2l - p) pi / p (Definition "grid"): the phase
    w (2l - p) pi / p is reduced exactly in integers."""
    w = grid.wavenumbers(p).astype(np.int64)[:, None]
    l = np.arange(p, dtype=np.int64)[None, :]
    r = w * (2 * l - p)                              # phase = pi r / p
    c = _cos_pi_ratio(r, p)
    s = _cos_pi_ratio(2 * r - p, 2 * p)            # sin(pi r / p) = cos(pi (2r - p) / (2p))
    return c + sign * 1j * s


def _cheb_forward_matrix(m):
    """DCT-I of Section 2 as a matrix: c_j = (2/(m-1)) w_j sum_a w_a f_a T_j(x_a),
    w = 1/2 at both ends, else 1 (discrete orthogonality of T_j at the
    Chebyshev extreme points)."""
    V = _cheb_at_grid(m)                     # V[a, j] = T_j(x_a)
    w = np.ones(m)
    w[0] = w[-1] = 0.5
    return (2.0 / (m - 1)) * (w[:, None] * (V * w[:, None]).T)


def _cheb_inverse_matrix(m):
    """Evaluation of a T-series at the grid: f_a = sum_j c_j T_j(x_a)."""
    return _cheb_at_grid(m)


def vals2coeffs_complex(f):
    """Values [p][m][n] (real or complex) -> full complex coefficients
    C[l][j][k] on wavenumber w = l - floor(p/2) (Section 2 transform order:
    r, then z, then theta)."""
    p, m, n = f.shape
    Wr = _cheb_forward_matrix(m)
    Wz = _cheb_forward_matrix(n)
    g = np.einsum('ja,lab->ljb', Wr, f)          # DCT-I along r
    g = np.einsum('kb,ljb->ljk', Wz, g)          # DCT-I along z
    E = _fourier_at_grid(p, -1) / p              # c_w = (1/p) sum_l f_l e^{-i w theta_l}
    return np.einsum('wl,ljk->wjk', E, g)


def coeffs2vals_complex(C):
    """Full complex coefficients -> values of the interpolant on the grid."""
    p, m, n = C.shape
    Vr = _cheb_inverse_matrix(m)
    Vz = _cheb_inverse_matrix(n)
    E = _fourier_at_grid(p, +1).T                # E[l, w] = e^{i w theta_l}
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


# ---------------------------------------------------------------- extended precision
# The same direct sums in np.longdouble (64-bit mantissa on x86, 112 on
# aarch64), with the matrices of the definitions built in that precision and
# every phase reduced exactly in integers.  Used to write reference values
# of computations whose FP64 rounding is amplified (the Navier-Stokes
# nonlinear term), never by the checks of the transforms themselves.
EXT = np.longdouble
PI_EXT = EXT('3.14159265358979323846264338327950288419716939937510')


def _cos_pi_ratio_ext(r, d):
    """cos(pi r / d) in extended precision, reduced as in ``_cos_pi_ratio``."""
    r = np.mod(np.asarray(r, dtype=np.int64), 2 * d)
    r = np.where(r > d, 2 * d - r, r)
    sign = np.where(2 * r > d, -1.0, 1.0).astype(EXT)
    r = np.where(2 * r > d, d - r, r)
    return sign * np.cos(PI_EXT * r.astype(EXT) / EXT(d))


def _cheb_at_grid_ext(m):
    N = m - 1
    a = np.arange(m, dtype=np.int64)[:, None]
    j = np.arange(m, dtype=np.int64)[None, :]
    return _cos_pi_ratio_ext(j * (N - a), N)


def _cheb_forward_matrix_ext(m):
    V = _cheb_at_grid_ext(m)
    w = np.ones(m, dtype=EXT)
    w[0] = w[-1] = EXT(0.5)
    return (EXT(2) / EXT(m - 1)) * (w[:, None] * (V * w[:, None]).T)


def _fourier_halfcomplex_ext(p):
    """Real matrices (F, I) of the theta stage in half-complex storage:
    F maps values over l to (c_0, Re c_1, Im c_1, ..., c_{-p/2}) with
    c_w = (1/p) sum_l f_l e^{-i w theta_l}; I maps them back,
    f_l = c_0 + 2 sum_w (Re c_w cos w theta_l - Im c_w sin w theta_l)
    + c_{-p/2} cos(p theta_l / 2) (theta_l = (2l - p) pi / p)."""
    l = np.arange(p, dtype=np.int64)
    F = np.zeros((p, p), dtype=EXT)
    I = np.zeros((p, p), dtype=EXT)

    def cos_sin(w):
        r = w * (2 * l - p)                              # phase pi r / p
        return _cos_pi_ratio_ext(r, p), _cos_pi_ratio_ext(2 * r - p, 2 * p)

    c, _ = cos_sin(0)
    F[0], I[:, 0] = c / p, c
    for w in range(1, p // 2):
        c, s = cos_sin(w)
        F[2 * w - 1], F[2 * w] = c / p, -s / p
        I[:, 2 * w - 1], I[:, 2 * w] = 2 * c, -2 * s
    c, _ = cos_sin(-(p // 2))
    F[p - 1], I[:, p - 1] = c / p, c
    return F, I


def vals2coeffs_ext(f):
    """``vals2coeffs`` in extended precision (input and output np.longdouble)."""
    p, m, n = f.shape
    g = np.einsum('ja,lab->ljb', _cheb_forward_matrix_ext(m), f)
    g = np.einsum('kb,ljb->ljk', _cheb_forward_matrix_ext(n), g)
    return np.einsum('wl,ljk->wjk', _fourier_halfcomplex_ext(p)[0], g)


def coeffs2vals_ext(H):
    """``coeffs2vals`` in extended precision."""
    p, m, n = H.shape
    g = np.einsum('lw,wjk->ljk', _fourier_halfcomplex_ext(p)[1], H)
    g = np.einsum('aj,ljk->lak', _cheb_at_grid_ext(m), g)
    return np.einsum('bk,lak->lab', _cheb_at_grid_ext(n), g)
