"""Pins of the oracle's grid and value <-> coefficient maps (Section 2)."""
import numpy as np
import pytest
from scipy import special

from oracle import grid, transforms as tr


@pytest.mark.parametrize('m', [4, 5, 9, 16])
def test_grid_definition(m):
    r = grid.cheb_points(m)
    assert r[0] == pytest.approx(-1.0) and r[-1] == pytest.approx(1.0)
    assert np.all(np.diff(r) > 0)
    assert np.allclose(r, -r[::-1], atol=1e-15)


@pytest.mark.parametrize('p', [2, 4, 8, 32])
def test_theta_grid_contains_antipodes(p):
    th = grid.theta_points(p)
    assert th[0] == pytest.approx(-np.pi)
    for t in th:
        assert np.min(np.abs(np.angle(np.exp(1j * (th - (t + np.pi)))))) < 1e-12
    assert list(grid.wavenumbers(p)) == list(range(-(p // 2), p - p // 2))


def _brute_values(C, r, z, th):
    """Interpolant of Section 2 evaluated by its defining triple sum."""
    p, m, n = C.shape
    w = grid.wavenumbers(p)
    Tr = np.array([special.eval_chebyt(j, r) for j in range(m)])      # [j][a]
    Tz = np.array([special.eval_chebyt(k, z) for k in range(n)])      # [k][b]
    E = np.exp(1j * np.outer(w, th))                                  # [wi][l]
    return np.einsum('wjk,ja,kb,wl->lab', C, Tr, Tz, E)


@pytest.mark.parametrize('p,m,n', [(4, 5, 6), (6, 7, 4), (8, 9, 9)])
def test_interpolation_identity(p, m, n):
    rng = np.random.default_rng(p * 100 + m * 10 + n)
    H = rng.standard_normal((p, m, n))
    v = tr.coeffs2vals(H)
    want = _brute_values(tr.halfcomplex_to_complex(H), grid.cheb_points(m), grid.cheb_points(n),
                         grid.theta_points(p))
    assert np.abs(want.imag).max() < 1e-12
    assert np.allclose(v, want.real, atol=1e-12)
    assert np.allclose(tr.vals2coeffs(v), H, atol=1e-12)


def _sample(fun, p, m, n):
    TH, RR, ZZ = np.meshgrid(grid.theta_points(p), grid.cheb_points(m), grid.cheb_points(n),
                             indexing='ij')
    return fun(RR, ZZ, TH)


def test_exp_z_chebyshev_closed_form():
    """e^x = I_0(1) + 2 sum_j I_j(1) T_j(x) pins the DCT-I normalisation."""
    p, m, n = 4, 5, 21
    H = tr.vals2coeffs(_sample(lambda r, z, t: np.exp(z) + 0 * r, p, m, n))
    want = np.array([special.iv(0, 1.0)] + [2.0 * special.iv(j, 1.0) for j in range(1, n)])
    assert np.allclose(H[0, 0, :], want, atol=1e-14)
    assert np.abs(H[1:]).max() < 1e-14 and np.abs(H[0, 1:]).max() < 1e-14
    H = tr.vals2coeffs(_sample(lambda r, z, t: np.exp(r) + 0 * z, p, 21, 5))
    assert np.allclose(H[0, :, 0], want, atol=1e-14)


def test_fourier_phase_and_layout():
    """x = r cos(theta) has c_{+-1} = T_1(r)/2; y = r sin(theta) has
    c_1 = -i T_1(r)/2; cos((p/2) theta) is the Nyquist basis function."""
    p, m, n = 8, 5, 4
    H = tr.vals2coeffs(_sample(lambda r, z, t: r * np.cos(t) + 0 * z, p, m, n))
    want = np.zeros((p, m, n)); want[1, 1, 0] = 0.5
    assert np.allclose(H, want, atol=1e-14)
    H = tr.vals2coeffs(_sample(lambda r, z, t: r * np.sin(t) + 0 * z, p, m, n))
    want = np.zeros((p, m, n)); want[2, 1, 0] = -0.5
    assert np.allclose(H, want, atol=1e-14)
    H = tr.vals2coeffs(_sample(lambda r, z, t: np.cos(p / 2 * t) + 0 * r * z, p, m, n))
    want = np.zeros((p, m, n)); want[p - 1, 0, 0] = 1.0
    assert np.allclose(H, want, atol=1e-14)


def test_bessel_generating_function():
    """e^{r cos theta} = sum_k I_k(r) e^{ik theta}: the k-th Fourier coefficient,
    summed back in r at the grid, is I_k(r_a) (aliasing below 1e-15 at p = 32)."""
    p, m, n = 32, 17, 4
    H = tr.vals2coeffs(_sample(lambda r, z, t: np.exp(r * np.cos(t)) + 0 * z, p, m, n))
    r = grid.cheb_points(m)
    T = np.array([special.eval_chebyt(j, r) for j in range(m)])
    for k, s in [(0, 0), (1, 1), (2, 3), (5, 9)]:
        assert np.allclose(H[s, :, 0] @ T, special.iv(k, r), atol=1e-14)      # Re c_k
        if k > 0:
            assert np.abs(H[s + 1, :, 0] @ T).max() < 1e-14                    # Im c_k = 0


def test_transform_matrices_accurate_at_high_degree():
    """At 512 points per axis the oracle's DCT-I entries T_j(x_a) and Fourier
    factors exp(-i w theta_l) agree with 40-digit evaluations (mpmath's own
    Chebyshev polynomials and exponential), entry by entry: a three-term
    recurrence or a floating-point phase w * theta_l drifts by ~1e-14 there,
    which would exceed the transforms' 1e-13 bar after summation."""
    mp = pytest.importorskip('mpmath')
    mp.mp.dps = 40
    L = 512
    V = tr._cheb_inverse_matrix(L)
    rng = np.random.default_rng(11)
    for a, j in [(0, 511), (1, 255), (100, 300), (255, 256), (511, 511)] + \
            [tuple(x) for x in rng.integers(0, L, size=(20, 2))]:
        x = mp.cos(mp.pi * (L - 1 - a) / (L - 1))
        assert abs(V[a, j] - float(mp.chebyt(int(j), x))) <= 4e-16
    p = 512
    E = tr._fourier_at_grid(p, -1)
    w = grid.wavenumbers(p)
    for wi, l in [(0, 511), (511, 3), (300, 300), (257, 100)] + [tuple(x) for x in rng.integers(0, p, size=(20, 2))]:
        th = mp.mpf(2 * int(l) - p) * mp.pi / p
        want = mp.exp(-1j * int(w[wi]) * th)
        assert abs(E[wi, l] - complex(want)) <= 4e-16
