"""Pins of the oracle's Poisson solve: manufactured solutions with the
Laplacian taken symbolically (sympy), tau exactness for polynomials, brute
force versus the QZ solver, and the parity structure of the doubled grid."""
import numpy as np
import pytest
import sympy as sp

from oracle import grid, heat, operators as ops, sylvester as sy, transforms as tr
from paper_2206_04827_gb300 import inputs

xs, ys, zs = sp.symbols('x y z')


def _laplacian_pair(expr):
    u = sp.lambdify((xs, ys, zs), expr, 'numpy')
    f = sp.lambdify((xs, ys, zs), -(sp.diff(expr, xs, 2) + sp.diff(expr, ys, 2) + sp.diff(expr, zs, 2)), 'numpy')
    return u, f


def _on_grid(fun, p, m, n):
    TH, RR, ZZ = np.meshgrid(grid.theta_points(p), grid.cheb_points(m), grid.cheb_points(n), indexing='ij')
    return fun(RR * np.cos(TH), RR * np.sin(TH), ZZ) + 0.0 * RR


POLY = (1 - xs ** 2 - ys ** 2) * (1 - zs ** 2) * (xs + ys ** 2 * zs)


@pytest.mark.parametrize('m,n,p', [(8, 7, 6), (9, 8, 8), (12, 10, 8), (17, 17, 16)])
def test_polynomial_solution_is_exact(m, n, p):
    """u is a CCF polynomial meeting the Dirichlet data: the tau solution
    equals it to rounding (no discretisation error at all)."""
    u, f = _laplacian_pair(POLY)
    Fc = tr.vals2coeffs(_on_grid(f, p, m, n))
    want = tr.vals2coeffs(_on_grid(u, p, m, n))
    assert np.abs(heat.poisson(Fc) - want).max() < 1e-13
    assert np.abs(heat.poisson(Fc, brute=True) - want).max() < 1e-13


def test_manufactured_forcing_closed_form():
    """inputs.manufactured_f is -lap u of inputs.manufactured_u (sympy)."""
    ex = (1 - xs ** 2 - ys ** 2) * (1 - zs ** 2) * sp.exp(xs + zs / 2)
    u, f = _laplacian_pair(ex)
    p, m, n = 6, 7, 5
    r, z, th = grid.cheb_points(m), grid.cheb_points(n), grid.theta_points(p)
    assert np.allclose(inputs.manufactured_u(r, z, th), _on_grid(u, p, m, n), atol=1e-13)
    assert np.allclose(inputs.manufactured_f(r, z, th), _on_grid(f, p, m, n), atol=1e-12)


def test_manufactured_exponential_spectral_accuracy():
    """The 33 x 33 x 32 manufactured problem: discrete solution within 1e-12
    of the interpolant of the exact u (spectral convergence)."""
    p, m, n = 32, 33, 33
    r, z, th = grid.cheb_points(m), grid.cheb_points(n), grid.theta_points(p)
    U = heat.poisson(tr.vals2coeffs(inputs.manufactured_f(r, z, th)))
    want = tr.vals2coeffs(inputs.manufactured_u(r, z, th))
    assert np.abs(U - want).max() / np.abs(want).max() < 1e-12


@pytest.mark.parametrize('m,n,k', [(6, 6, 0), (7, 8, 1), (9, 7, 3), (10, 10, 5)])
def test_brute_force_equals_qz(m, n, k):
    rng = np.random.default_rng(7 + k)
    for kind, ka in [('poisson', None), ('heat', 0.37)]:
        ms = sy.ModeSystem(m, n, k, kind, ka)
        E = rng.standard_normal((m - 2, n - 2))
        Yk = sy.solve_kron(ms.A, ms.B, ms.C, ms.D, E)
        Yb = sy.BartelsStewart(ms.A, ms.B, ms.C, ms.D).solve(E)
        assert np.abs(Yk - Yb).max() < 1e-11 * np.abs(Yk).max()
        assert np.abs(ms.apply(Yb) - E).max() < 1e-11 * np.abs(E).max()


def test_parity_blocks_decouple():
    """All operators have even bandwidth offsets, and a real field on the
    doubled grid has c_{i,j,k} = 0 unless i = k (mod 2): the Poisson solution
    keeps that structure."""
    p, m, n = 8, 11, 9
    for k in range(5):
        for M in sy.ModeSystem(m, n, k, 'heat', 0.3).__dict__.values():
            if isinstance(M, np.ndarray) and M.ndim == 2 and M.shape[0] == M.shape[1]:
                i, j = np.nonzero(np.abs(M) > 0)
                assert np.all((i - j) % 2 == 0)
    F = inputs.smooth_coeffs(p, m, n, 1.3, np.random.default_rng(1))
    U = heat.poisson(F)
    for s in range(p):
        k = tr.slice_wavenumber(s, p)
        assert np.abs(U[s, (1 - k % 2)::2, :]).max() == 0.0


def test_planted_operator_error_is_caught():
    """A plausible oracle mistake (R's sub- and superdiagonal swapped) breaks
    the polynomial pin: the pins can see such errors."""
    u, f = _laplacian_pair(POLY)
    p, m, n = 8, 9, 8
    Fc = tr.vals2coeffs(_on_grid(f, p, m, n))
    want = tr.vals2coeffs(_on_grid(u, p, m, n))
    good = ops.mult_r_C2
    try:
        ops.mult_r_C2 = lambda mm: good(mm).T
        bad = heat.poisson(Fc)
    finally:
        ops.mult_r_C2 = good
    assert np.abs(bad - want).max() > 1e-3
