"""Pins of the CPU ADI (oracle/adi.py, Algorithm 1 with the shifts of
Section 3) against what the mathematics fixes: the Moebius map takes all four
points -alpha, -1, 1, alpha to a, b, c, d (the fourth is implied by alpha's
formula); the product of the per-iteration error factors stays below the
tolerance on the whole spectral rectangle (the Zolotarev bound the shift
choice is made for); on diagonal matrices the iterate after J steps is the
exact solution times one minus that product, element by element; and the
iteration reaches the direct (QZ) solve of the same equations."""
import types

import numpy as np
import pytest

from oracle import adi, heat as oheat
from oracle.sylvester import ModeSystem
from paper_2206_04827_gb300 import inputs


def _factor(lam, mu, p, q):
    r = np.ones(np.broadcast(lam, mu).shape)
    for pj, qj in zip(p, q):
        r = r * (lam - qj) * (mu - pj) / ((lam - pj) * (mu - qj))
    return r


@pytest.mark.parametrize('a,b,c,d', [(1.0, 50.0, -40.0, -0.01), (0.3, 2e4, -3e3, -2.5), (1.0, 1.2, -9.0, -0.5)])
def test_mobius_takes_all_four_points(a, b, c, d):
    J, p, q, gamma, alpha, T = adi.zolotarev_shifts(a, b, c, d, 1e-12)
    got = T(np.array([-alpha, -1.0, 1.0, alpha]))
    assert np.allclose(got, [a, b, c, d], rtol=1e-9, atol=0)
    assert gamma > 1 and alpha > 1
    assert np.all((q >= a) & (q <= b)) and np.all((p >= c) & (p <= d))


@pytest.mark.parametrize('tol', [1e-6, 1e-10, 1e-14])
@pytest.mark.parametrize('a,b,c,d', [(1.0, 66.4, -43.9, -0.0033), (0.5, 3e3, -2e5, -1.1)])
def test_shifts_meet_the_tolerance_on_the_spectral_rectangle(a, b, c, d, tol):
    J, p, q, _, _, _ = adi.zolotarev_shifts(a, b, c, d, tol)
    # geometric grids reach both ends of intervals spanning decades
    lam = np.geomspace(a, b, 1501)[:, None]
    mu = -np.geomspace(-c, -d, 1501)[None, :]
    assert np.abs(_factor(lam, mu, p, q)).max() <= tol


def test_diagonal_iterate_is_the_solution_times_one_minus_the_factor():
    lam = np.array([1.5, 7.0, 40.0, 200.0])
    mu = np.array([-300.0, -20.0, -2.0, -0.1, -0.02])
    ms = types.SimpleNamespace(A=np.diag(lam), C=np.eye(4), B=np.eye(5), D=np.diag(-mu))
    E = np.random.default_rng(0).standard_normal((4, 5))
    X = E / (lam[:, None] - mu[None, :])                   # A X B^T + C X D^T = E
    J, p, q, _, _, _ = adi.zolotarev_shifts(lam.min(), lam.max(), mu.min(), mu.max(), 1e-5)
    XJ = adi.adi_solve(ms, E, p, q)
    want = X * (1.0 - _factor(lam[:, None], mu[None, :], p, q))
    assert np.abs(XJ - want).max() <= 1e-13 * np.abs(X).max()
    assert 0 < np.abs(XJ - X).max() <= 1e-5 * np.abs(X).max() * 10


@pytest.mark.parametrize('kind', ['poisson', 'heat'])
def test_interval_ends_bracket_the_pencil_spectra(kind):
    ka = 2e-3 if kind == 'heat' else None
    ms = ModeSystem(30, 27, 4, kind, ka)
    a, b, c, d = adi.spectral_intervals(ms, kind, ka)
    lam = np.real(np.linalg.eigvals(np.linalg.solve(ms.C, ms.A)))
    mu = np.real(np.linalg.eigvals(-ms.D @ np.linalg.inv(ms.B)))
    assert a < lam.min() and lam.max() < b and c < mu.min() and mu.max() < d


@pytest.mark.parametrize('p,m,n', [(4, 24, 21), (6, 40, 37)])
def test_adi_reaches_the_direct_solve(p, m, n):
    rng = np.random.default_rng(m + n)
    F = inputs.smooth_coeffs(p, m, n, 1.2, rng)
    g = inputs.smooth_coeffs(p, m, n, 1.25, rng)
    u, w = adi.poisson(F, 1e-14), oheat.poisson(F)
    assert np.abs(u - w).max() <= 1e-12 * np.abs(w).max()
    h, w = adi.heat_steps(F, g, 0.7, 2e-3, 3, 1e-14), oheat.heat_steps(F, g, 0.7, 2e-3, 3)
    assert np.abs(h - w).max() <= 1e-12 * np.abs(w).max()
    # a loose tolerance stops early, as the bound says
    u6 = adi.poisson(F, 1e-6)
    assert 1e-12 < np.abs(u6 - oheat.poisson(F)).max() / np.abs(w).max() < 1e-4
