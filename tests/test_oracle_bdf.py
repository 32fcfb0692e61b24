"""Pins of the oracle's higher-order BDF (Section 3, BDF 1 / BDF 4 and the
delta^(b), kappa^(b) definitions): the printed BDF 4 coefficients, exactness
of every order on polynomials in t, the scalar recurrence of a Dirichlet
eigenmode (start-up through lower orders included), the temporal order of
convergence, and BDF 1 = the BDF1 stepper."""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import grid, heat, transforms as tr
from paper_2206_04827_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), 'golden', 'bdf4_printed.txt')


def _printed():
    vals = {}
    with open(GOLD) as fh:
        for line in fh:
            line = line.split('#')[0].split()
            if line:
                vals[line[0]] = Fraction(line[1])
    return vals


def test_bdf4_matches_printed_coefficients():
    kap, beta = heat.bdf_coefficients(4)
    pr = _printed()
    assert kap == pr['kappa']
    assert beta == [pr['beta0'], pr['beta1'], pr['beta2'], pr['beta3']]


@pytest.mark.parametrize('b', [1, 2, 3, 4])
def test_bdf_is_exact_on_polynomials_in_time(b):
    """y(t) = t^q, q <= b: y(t+h) - kappa h y'(t+h) = sum beta_i y(t - i h)
    holds exactly (the definition of order b); q = b + 1 fails."""
    kap, beta = heat.bdf_coefficients(b)
    h, t = Fraction(1, 3), Fraction(5, 7)
    for q in range(b + 2):
        lhs = (t + h) ** q - kap * h * (q * (t + h) ** (q - 1) if q else 0)
        rhs = sum(beta[i] * (t - i * h) ** q for i in range(b))
        assert (lhs == rhs) == (q <= b)


def test_bdf1_run_is_the_bdf1_stepper():
    p, m, n = 6, 9, 8
    rng = np.random.default_rng(3)
    X0 = inputs.smooth_coeffs(p, m, n, 1.3, rng)
    g = np.stack([inputs.smooth_coeffs(p, m, n, 1.3, rng) for _ in range(3)])
    a = heat.heat_bdf(X0[None], g, 0.7, 0.02, 1, 3)[0]
    b = heat.heat_steps(X0, g, 0.7, 0.02, 3)
    assert np.abs(a - b).max() == 0.0


def _eigen(p, m, n, mu, nu, trig):
    r, z, th = grid.cheb_points(m), grid.cheb_points(n), grid.theta_points(p)
    return tr.vals2coeffs(inputs.eigenmode_values(r, z, th, [(mu, nu, trig, 1.0)])), inputs.eigenvalue(mu, nu)


@pytest.mark.parametrize('order,nvalid', [(2, 1), (3, 1), (4, 1), (4, 2), (4, 4)])
def test_eigenmode_follows_scalar_recurrence(order, nvalid):
    """For a Dirichlet eigenmode E with eigenvalue lambda, each step scales by
    the scalar BDF recurrence a_{s+1} (1 + kappa_b alpha lambda) = sum beta_i
    a_{s-i}, b = min(order, known states): the field stays a_s E up to the
    spatial (spectral) error."""
    p, m, n = 8, 33, 33
    alpha, h, steps = 0.8, 0.01, 6
    E, lam = _eigen(p, m, n, 1, 1, 0)
    a0 = [1.0, 1.1, 1.25, 1.4][:nvalid]
    hist = np.zeros((order, p, m, n))
    for i, ai in enumerate(a0):
        hist[i] = ai * E
    out = heat.heat_bdf(hist, np.zeros((p, m, n)), alpha, h, order, steps, nvalid=nvalid)
    amps = list(a0)                                   # newest first
    for _ in range(steps):
        b = min(order, len(amps))
        kap, beta = heat.bdf_coefficients(b)
        nxt = sum(float(beta[i]) * amps[i] for i in range(b)) / (1 + float(kap) * h * alpha * lam)
        amps = [nxt] + amps[:order - 1]
    for i, ai in enumerate(amps):
        assert np.abs(out[i] - ai * E).max() < 1e-12 * np.abs(E).max()


@pytest.mark.parametrize('order', [2, 3, 4])
def test_temporal_order_of_convergence(order):
    """Exact history exp(-alpha lambda t) of an eigenmode: the error at a fixed
    time falls like h^order (ratio 2^order when h halves)."""
    p, m, n = 8, 25, 25
    alpha, T = 1.0, 0.2
    E, lam = _eigen(p, m, n, 0, 1, 0)
    errs = []
    for steps in (10, 20):
        h = T / steps
        hist = np.stack([np.exp(alpha * lam * i * h) * E for i in range(order)])  # X_0 = E, X_{-i}
        out = heat.heat_bdf(hist, np.zeros((p, m, n)), alpha, h, order, steps)
        errs.append(np.abs(out[0] - np.exp(-alpha * lam * T) * E).max())
    rate = np.log2(errs[0] / errs[1])
    assert abs(rate - order) < 0.35, (errs, rate)


def test_lifting_in_bdf_run():
    """With non-zero wall data, a BDF 3 run of a polynomial steady state u
    (forcing g = -alpha lap u, every history slot u) stays at u exactly."""
    import sympy as sp
    xs, ys, zs = sp.symbols('x y z')
    u = (xs ** 2 + ys * zs + 2) * (1 + zs ** 2)
    gx = -0.5 * (sp.diff(u, xs, 2) + sp.diff(u, ys, 2) + sp.diff(u, zs, 2))
    p, m, n = 8, 9, 8
    TH, RR, ZZ = np.meshgrid(grid.theta_points(p), grid.cheb_points(m), grid.cheb_points(n), indexing='ij')
    ev = lambda e: sp.lambdify((xs, ys, zs), e, 'numpy')(RR * np.cos(TH), RR * np.sin(TH), ZZ) + 0.0 * RR
    uv, G = ev(u), tr.vals2coeffs(ev(gx))
    U = tr.vals2coeffs(uv)
    out = heat.heat_bdf(np.stack([U] * 3), G, 0.5, 0.1, 3, 4, bc=uv)
    assert np.abs(out - U[None]).max() < 1e-12 * np.abs(U).max()


def _bdf_problem(order, nvalid, steps, seed, p=4, m=7, n=6, varying=True):
    rng = np.random.default_rng(seed)
    hist = np.zeros((order, p, m, n))
    for i in range(nvalid):
        hist[i] = inputs.smooth_coeffs(p, m, n, 1.3, rng)
    g = (np.stack([inputs.smooth_coeffs(p, m, n, 1.3, rng) for _ in range(steps)]) if varying
         else inputs.smooth_coeffs(p, m, n, 1.3, rng))
    tgt = np.stack([inputs.smooth_coeffs(p, m, n, 1.3, rng) for _ in range(order)])
    return hist, g, tgt


@pytest.mark.parametrize('order,nvalid,steps,varying,wall', [(2, 1, 4, True, False), (4, 1, 6, False, False),
                                                             (4, 3, 3, True, True), (3, 3, 2, True, False),
                                                             (4, 4, 2, False, False)])
def test_bdf_adjoint_matches_central_differences(order, nvalid, steps, varying, wall):
    """L = sum over the final history of |X - target|^2 (only the known
    slots): gradients w.r.t. the initial history, g and alpha against central
    differences of the forward run."""
    alpha, dt = 0.6, 0.02
    hist, g, tgt = _bdf_problem(order, nvalid, steps, 40 + order + nvalid, varying=varying)
    bc = tr.coeffs2vals(inputs.smooth_coeffs(4, 7, 6, 1.1, np.random.default_rng(1))) if wall else None
    keep = min(order, nvalid + steps)

    def loss(h_, g_, a_):
        out = heat.heat_bdf(h_, g_, a_, dt, order, steps, nvalid=nvalid, bc=bc)
        return float(np.sum((out[:keep] - tgt[:keep]) ** 2))

    out = heat.heat_bdf(hist, g, alpha, dt, order, steps, nvalid=nvalid, bc=bc)
    dout = np.zeros_like(out)
    dout[:keep] = 2.0 * (out[:keep] - tgt[:keep])
    dh, dg, dal = heat.heat_bdf_adjoint(hist, g, alpha, dt, order, steps, dout, nvalid=nvalid, bc=bc)
    rng = np.random.default_rng(5)
    h = 1e-3
    d = np.zeros_like(hist)
    d[:nvalid] = rng.standard_normal(hist[:nvalid].shape)
    fd = (loss(hist + h * d, g, alpha) - loss(hist - h * d, g, alpha)) / (2 * h)
    assert abs(fd - float(np.sum(dh * d))) <= 1e-7 * abs(fd)
    assert np.all(dh[nvalid:] == 0.0)
    d = rng.standard_normal(g.shape)
    fd = (loss(hist, g + h * d, alpha) - loss(hist, g - h * d, alpha)) / (2 * h)
    assert abs(fd - float(np.sum(dg * d))) <= 1e-7 * abs(fd)
    ha = 1e-4 * alpha
    fd = (loss(hist, g, alpha + ha) - loss(hist, g, alpha - ha)) / (2 * ha)
    assert abs(fd - dal) <= 1e-7 * abs(fd)


def test_bdf_adjoint_is_dense_transpose():
    """Assemble the linear map (initial history) -> (final history) of a BDF 3
    run with start-up column by column; the adjoint applied to c equals
    Phi^T c."""
    order, nvalid, steps = 3, 2, 4
    hist, g, _ = _bdf_problem(order, nvalid, steps, 9, p=2, m=6, n=5)
    zero_g = np.zeros_like(g)
    shape = hist[:nvalid].shape
    size_in = int(np.prod(shape))
    cols = []
    for col in range(size_in):
        e = np.zeros(size_in); e[col] = 1.0
        h0 = np.zeros_like(hist); h0[:nvalid] = e.reshape(shape)
        cols.append(heat.heat_bdf(h0, zero_g, 0.5, 0.03, order, steps, nvalid=nvalid).ravel())
    Phi = np.array(cols).T
    c = np.random.default_rng(3).standard_normal(hist.shape)
    dh, _, _ = heat.heat_bdf_adjoint(hist, zero_g, 0.5, 0.03, order, steps, c, nvalid=nvalid)
    assert np.allclose(dh[:nvalid].ravel(), Phi.T @ c.ravel(), atol=1e-12 * np.abs(Phi).max())
