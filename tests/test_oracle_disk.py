"""Pins of the oracle's horizontal (disk) Poisson solve (Section 4, eq.
ptpoisson): tau exactness on polynomials that vanish on the wall (horizontal
Laplacian by sympy), Bessel x arbitrary-z eigenfunctions of -Delta_h to
spectral accuracy, and the independence of the z columns."""
import numpy as np
import pytest
import sympy as sp
from scipy import special

from oracle import disk, grid, transforms as tr
from paper_2206_04827_gb300 import inputs

xs, ys, zs = sp.symbols('x y z')


def _on_grid(fun, p, m, n):
    TH, RR, ZZ = np.meshgrid(grid.theta_points(p), grid.cheb_points(m), grid.cheb_points(n), indexing='ij')
    return fun(RR * np.cos(TH), RR * np.sin(TH), ZZ) + 0.0 * RR


@pytest.mark.parametrize('m,n,p', [(9, 6, 8), (12, 9, 10), (15, 5, 12)])
def test_polynomial_solution_is_exact(m, n, p):
    """u = (1 - x^2 - y^2)(x + y^2 z + x y z^3 + 2): -Delta_h u by sympy; the tau
    solution reproduces u to rounding (u vanishes on the wall only, not at
    z = +-1: the z direction carries no condition)."""
    u = (1 - xs ** 2 - ys ** 2) * (xs + ys ** 2 * zs + xs * ys * zs ** 3 + 2)
    f = -(sp.diff(u, xs, 2) + sp.diff(u, ys, 2))
    U = tr.vals2coeffs(_on_grid(sp.lambdify((xs, ys, zs), u, 'numpy'), p, m, n))
    Fc = tr.vals2coeffs(_on_grid(sp.lambdify((xs, ys, zs), f, 'numpy'), p, m, n))
    assert np.abs(disk.horizontal_poisson(Fc) - U).max() < 1e-13 * np.abs(U).max()


@pytest.mark.parametrize('mu,nu', [(0, 1), (1, 1), (2, 2), (3, 1)])
def test_bessel_eigenfunctions(mu, nu):
    """u = J_mu(j r) cos(mu theta) exp(z) with J_mu(j) = 0 satisfies
    -Delta_h u = j^2 u: the discrete solution matches u to spectral
    accuracy."""
    p, m, n = 16, 33, 9
    j = special.jn_zeros(mu, nu)[-1]
    TH, RR, ZZ = np.meshgrid(grid.theta_points(p), grid.cheb_points(m), grid.cheb_points(n), indexing='ij')
    u = special.jv(mu, j * RR) * np.cos(mu * TH) * np.exp(ZZ)
    U = disk.horizontal_poisson(tr.vals2coeffs(j ** 2 * u))
    assert np.abs(tr.coeffs2vals(U) - u).max() < 1e-11 * np.abs(u).max()


def test_z_columns_are_independent():
    rng = np.random.default_rng(4)
    p, m, n = 6, 11, 7
    F = rng.standard_normal((p, m, n))
    full = disk.horizontal_poisson(F)
    for col in (0, 3, 6):
        Fc = np.zeros_like(F)
        Fc[:, :, col] = F[:, :, col]
        part = disk.horizontal_poisson(Fc)
        assert np.abs(part[:, :, col] - full[:, :, col]).max() < 1e-13 * np.abs(full).max()
        others = np.delete(part, col, axis=2)
        assert np.abs(others).max() == 0.0


def test_wall_values_vanish():
    rng = np.random.default_rng(8)
    p, m, n = 8, 13, 6
    U = disk.horizontal_poisson(inputs.smooth_coeffs(p, m, n, 1.2, rng))
    V = tr.coeffs2vals(U)
    assert np.abs(V[:, [0, -1], :]).max() < 1e-14 * np.abs(V).max()
