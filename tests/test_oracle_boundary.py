"""Pins of the oracle's non-zero Dirichlet data (lifting): polynomial
solutions with non-zero wall values are reproduced exactly, a harmonic
function is recovered from its boundary values alone, lifting equals the
bordered tau system (boundary rows appended, no recombined basis) for
arbitrary data, and the blend reproduces bilinear data everywhere."""
import numpy as np
import pytest
import sympy as sp

from oracle import grid, heat, transforms as tr

xs, ys, zs = sp.symbols('x y z')


def _on_grid(fun, p, m, n):
    TH, RR, ZZ = np.meshgrid(grid.theta_points(p), grid.cheb_points(m), grid.cheb_points(n), indexing='ij')
    return fun(RR * np.cos(TH), RR * np.sin(TH), ZZ) + 0.0 * RR


def _fun(expr):
    return sp.lambdify((xs, ys, zs), expr, 'numpy')


def _lap(expr):
    return sp.diff(expr, xs, 2) + sp.diff(expr, ys, 2) + sp.diff(expr, zs, 2)


WALLY = (xs ** 2 + ys * zs + 2) * (1 + zs ** 2) * (3 + xs * ys)


@pytest.mark.parametrize('m,n,p', [(9, 8, 10), (12, 11, 8), (14, 9, 12)])
def test_polynomial_with_wall_values_is_exact(m, n, p):
    """u is a polynomial that does not vanish on the wall: with its own grid
    values as boundary data the tau solution equals it to rounding, both by
    lifting + Bartels-Stewart and by the bordered dense system."""
    u = _on_grid(_fun(WALLY), p, m, n)
    F = tr.vals2coeffs(_on_grid(_fun(-_lap(WALLY)), p, m, n))
    want = tr.vals2coeffs(u)
    scale = np.abs(want).max()
    assert np.abs(heat.poisson(F, bc=u) - want).max() < 1e-13 * scale
    assert np.abs(heat.poisson(F, bc=u, brute=True) - want).max() < 1e-13 * scale


def test_interior_of_bc_array_is_ignored():
    """Only the boundary nodes of the bc array are data."""
    p, m, n = 8, 9, 8
    u = _on_grid(_fun(WALLY), p, m, n)
    F = tr.vals2coeffs(_on_grid(_fun(-_lap(WALLY)), p, m, n))
    noisy = u.copy()
    noisy[:, 1:-1, 1:-1] = np.random.default_rng(3).standard_normal((p, m - 2, n - 2))
    assert np.abs(heat.poisson(F, bc=noisy) - heat.poisson(F, bc=u)).max() < 1e-13


def test_harmonic_function_from_boundary_values():
    """u = exp(z) cos(x) is harmonic: with f = 0 the solution is determined by
    the wall data alone and converges spectrally to u."""
    expr = sp.exp(zs) * sp.cos(xs)
    assert sp.simplify(_lap(expr)) == 0
    p, m, n = 24, 25, 25
    u = _on_grid(_fun(expr), p, m, n)
    U = heat.poisson(np.zeros((p, m, n)), bc=u)
    assert np.abs(tr.coeffs2vals(U) - u).max() < 1e-12


@pytest.mark.parametrize('m,n,p', [(7, 6, 4), (8, 9, 6)])
def test_lifting_equals_bordered_system_for_arbitrary_data(m, n, p):
    """Random right side and random (rough) wall values: the lifted solve and
    the bordered tau system are the same discrete problem, for the Poisson
    equation and for one BDF1 step."""
    rng = np.random.default_rng(11)
    F = rng.standard_normal((p, m, n))
    bc = rng.standard_normal((p, m, n))
    a = heat.poisson(F, bc=bc)
    b = heat.poisson(F, bc=bc, brute=True)
    assert np.abs(a - b).max() < 1e-10 * np.abs(a).max()
    X0 = rng.standard_normal((p, m, n))
    a = heat.heat_steps(X0, F, 0.8, 0.03, 1, bc=bc)
    b = heat.heat_steps(X0, F, 0.8, 0.03, 1, bc=bc, brute=True)
    assert np.abs(a - b).max() < 1e-10 * np.abs(a).max()


def test_solution_traces_equal_the_data():
    """The solution's values on the four faces of every theta slice equal the
    data there (the corner values are consistent because they come from one
    function)."""
    rng = np.random.default_rng(5)
    p, m, n = 6, 10, 9
    bc = tr.coeffs2vals(rng.standard_normal((p, m, n)))
    Uv = tr.coeffs2vals(heat.poisson(rng.standard_normal((p, m, n)), bc=bc))
    for sl in (np.s_[:, 0, :], np.s_[:, -1, :], np.s_[:, :, 0], np.s_[:, :, -1]):
        assert np.abs(Uv[sl] - bc[sl]).max() < 1e-12 * np.abs(bc).max()


def test_blend_reproduces_bilinear_data():
    """The transfinite blend of data that is bilinear in (r, z) on every slice
    is that data everywhere."""
    p, m, n = 4, 7, 6
    r = grid.cheb_points(m)[None, :, None]
    z = grid.cheb_points(n)[None, None, :]
    c = np.arange(1, p + 1, dtype=float)[:, None, None]
    vals = c * (1.0 + 0.3 * r - 0.7 * z + 0.2 * r * z) + 0.0 * r * z
    assert np.abs(tr.coeffs2vals(heat.lifting(vals)) - vals).max() < 1e-14


def test_zero_data_is_the_homogeneous_solve():
    rng = np.random.default_rng(2)
    F = rng.standard_normal((6, 9, 8))
    assert np.abs(heat.poisson(F, bc=np.zeros((6, 9, 8))) - heat.poisson(F)).max() < 1e-15


def test_heat_step_with_wall_values_is_exact():
    """X1 = u (non-zero on the wall, data = u's traces), X0 = v arbitrary
    polynomial, g = (u - h alpha lap u - v) / h: one BDF1 step returns u."""
    alpha, h = 0.6, 0.04
    u = WALLY
    v = (1 + xs * zs) * (2 - ys ** 2)
    g = (u - h * alpha * _lap(u) - v) / h
    p, m, n = 8, 9, 8
    U, V, G = (tr.vals2coeffs(_on_grid(_fun(e), p, m, n)) for e in (u, v, g))
    uv = _on_grid(_fun(u), p, m, n)
    for brute in (False, True):
        X1 = heat.heat_steps(V, G, alpha, h, 1, brute=brute, bc=uv)
        assert np.abs(X1 - U).max() < 1e-13 * np.abs(U).max()
