"""Pins of the oracle's BDF1 heat stepping (Section 3, BDF 1 and eq.
HelmholtzMatEqn): exact polynomial steps, Bessel x sine eigenmode decay
(1 + alpha h lambda)^-s, the continuous decay exp(-alpha lambda t) to O(h),
and the Poisson steady state."""
import numpy as np
import pytest
import sympy as sp

from oracle import grid, heat, transforms as tr
from paper_2206_04827_gb300 import inputs

xs, ys, zs = sp.symbols('x y z')


def _on_grid(fun, p, m, n):
    TH, RR, ZZ = np.meshgrid(grid.theta_points(p), grid.cheb_points(m), grid.cheb_points(n), indexing='ij')
    return fun(RR * np.cos(TH), RR * np.sin(TH), ZZ) + 0.0 * RR


def test_polynomial_step_is_exact():
    """Choose X1 = u and X0 = v (polynomials meeting the Dirichlet data) and
    g = (u - h alpha lap u - v) / h: one BDF1 step must return u exactly."""
    alpha, h = 0.7, 0.05
    u = (1 - xs ** 2 - ys ** 2) * (1 - zs ** 2) * (xs * zs + ys ** 2)
    v = (1 - xs ** 2 - ys ** 2) * (1 - zs ** 2) * (1 + xs * ys)
    lap = sp.diff(u, xs, 2) + sp.diff(u, ys, 2) + sp.diff(u, zs, 2)
    g = (u - h * alpha * lap - v) / h
    p, m, n = 8, 9, 8
    U, V, G = (tr.vals2coeffs(_on_grid(sp.lambdify((xs, ys, zs), e, 'numpy'), p, m, n)) for e in (u, v, g))
    for brute in (False, True):
        X1 = heat.heat_steps(V, G, alpha, h, 1, brute=brute)
        assert np.abs(X1 - U).max() < 1e-13


@pytest.mark.parametrize('mu,nu,trig', [(0, 1, 0), (1, 1, 0), (2, 1, 1), (1, 2, 0)])
def test_eigenmode_discrete_decay(mu, nu, trig):
    """For a Dirichlet eigenmode with eigenvalue lambda = j_{mu,nu}^2 + (nu pi/2)^2,
    BDF1 multiplies the field by exactly 1/(1 + alpha h lambda) per step, up
    to the (spectrally small) spatial error."""
    p, m, n = 8, 33, 33
    alpha, h, s = 1.0, 1e-3, 5
    r, z, th = grid.cheb_points(m), grid.cheb_points(n), grid.theta_points(p)
    X0 = tr.vals2coeffs(inputs.eigenmode_values(r, z, th, [(mu, nu, trig, 1.0)]))
    Xs = heat.heat_steps(X0, np.zeros_like(X0), alpha, h, s)
    fac = (1.0 + alpha * h * inputs.eigenvalue(mu, nu)) ** (-s)
    assert np.abs(Xs - fac * X0).max() / np.abs(X0).max() < 1e-12


def test_eigenmode_continuous_decay_first_order():
    """exp(-alpha lambda t) is matched to O(h): the error halves with h."""
    p, m, n = 4, 25, 25
    alpha, T = 1.0, 0.02
    r, z, th = grid.cheb_points(m), grid.cheb_points(n), grid.theta_points(p)
    X0 = tr.vals2coeffs(inputs.eigenmode_values(r, z, th, [(0, 1, 0, 1.0)]))
    lam = inputs.eigenvalue(0, 1)
    errs = []
    for steps in (10, 20):
        Xs = heat.heat_steps(X0, np.zeros_like(X0), alpha, T / steps, steps)
        errs.append(np.abs(Xs - np.exp(-alpha * lam * T) * X0).max() / np.abs(X0).max())
    assert errs[0] < 0.05
    assert 1.8 < errs[0] / errs[1] < 2.2


def test_large_step_reaches_poisson_steady_state():
    """BDF1 is L-stable: one step of size h -> infinity from X0 = 0 with
    forcing g gives the steady state -alpha lap X = g, the Poisson solution
    with f = g / alpha."""
    p, m, n = 6, 9, 8
    alpha = 0.5
    G = inputs.smooth_coeffs(p, m, n, 1.4, np.random.default_rng(5))
    X = heat.heat_steps(np.zeros_like(G), G, alpha, 1e9, 1)
    U = heat.poisson(G / alpha)
    assert np.abs(X - U).max() < 1e-7 * np.abs(U).max()


@pytest.mark.parametrize('m', [128, 256])
def test_refinement_recovers_exact_polynomial_step_on_large_grids(m):
    """One BDF1 step whose exact discrete solution is a known polynomial u
    (tau-exact), on a large grid with a small kappa*alpha (the 512^3
    workload's 1e-5): one step of iterative refinement with an extended
    precision residual brings the direct solve to ~1e-14 (the plain QZ solve
    drifts to ~1e-12 at m = 256)."""
    alpha, h = 0.1, 1e-4
    u = (1 - xs ** 2 - ys ** 2) * (1 - zs ** 2) * (xs * zs + ys ** 2 + 2)
    v = (1 - xs ** 2 - ys ** 2) * (1 - zs ** 2) * (1 + xs * ys)
    lap = sp.diff(u, xs, 2) + sp.diff(u, ys, 2) + sp.diff(u, zs, 2)
    g = (u - h * alpha * lap - v) / h
    p = 6
    U, V, G = (tr.vals2coeffs(_on_grid(sp.lambdify((xs, ys, zs), e, 'numpy'), p, m, m)) for e in (u, v, g))
    sl = [0, 1, 2]
    X0 = heat.heat_steps(V, G, alpha, h, 1, slices=sl)
    X1 = heat.heat_steps(V, G, alpha, h, 1, slices=sl, refine=1)
    scale = np.abs(U).max()
    e0 = np.abs(X0[sl] - U[sl]).max() / scale
    e1 = np.abs(X1[sl] - U[sl]).max() / scale
    assert e1 < 3e-14 and e1 <= e0
