"""Pins of the oracle's discrete adjoint: central finite differences and the
dense transpose of the assembled step map."""
import numpy as np

from oracle import heat
from paper_2206_04827_gb300 import inputs

P, M, N = 4, 7, 6
ALPHA, DT, STEPS = 0.6, 0.01, 3


def _problem(seed=0):
    rng = np.random.default_rng(seed)
    X0 = inputs.smooth_coeffs(P, M, N, 1.3, rng)
    g = np.stack([inputs.smooth_coeffs(P, M, N, 1.3, rng) for _ in range(STEPS)])
    tgt = inputs.smooth_coeffs(P, M, N, 1.3, rng)
    return X0, g, tgt


def _loss(X0, g, alpha):
    XN = heat.heat_steps(X0, g, alpha, DT, STEPS)
    return float(np.sum((XN - _problem()[2]) ** 2))


def test_gradients_match_central_differences():
    X0, g, tgt = _problem()
    XN = heat.heat_steps(X0, g, ALPHA, DT, STEPS)
    dX0, dg, dal = heat.heat_adjoint(X0, g, ALPHA, DT, STEPS, 2.0 * (XN - tgt))
    rng = np.random.default_rng(11)
    for which in ('X0', 'g'):
        d = rng.standard_normal(X0.shape if which == 'X0' else g.shape)
        h = 1e-3
        if which == 'X0':
            fd = (_loss(X0 + h * d, g, ALPHA) - _loss(X0 - h * d, g, ALPHA)) / (2 * h)
            an = float(np.sum(dX0 * d))
        else:
            fd = (_loss(X0, g + h * d, ALPHA) - _loss(X0, g - h * d, ALPHA)) / (2 * h)
            an = float(np.sum(dg * d))
        assert abs(fd - an) <= 1e-7 * max(abs(fd), 1e-300)
    h = 1e-4 * ALPHA
    fd = (_loss(X0, g, ALPHA + h) - _loss(X0, g, ALPHA - h)) / (2 * h)
    assert abs(fd - dal) <= 1e-7 * abs(fd)


def test_dense_transpose_of_step_map():
    """Assemble X_N = Phi X_0 column by column (unit inputs); dL/dX0 for
    L = <c, X_N> must be Phi^T c."""
    X0, g, _ = _problem(1)
    zero_g = np.zeros_like(g)
    n = X0.size
    Phi = np.zeros((n, n))
    for col in range(n):
        e = np.zeros(n); e[col] = 1.0
        Phi[:, col] = heat.heat_steps(e.reshape(X0.shape), zero_g, ALPHA, DT, STEPS).ravel()
    c = np.random.default_rng(2).standard_normal(X0.shape)
    dX0, dg, _ = heat.heat_adjoint(X0, zero_g, ALPHA, DT, STEPS, c)
    assert np.allclose(dX0.ravel(), Phi.T @ c.ravel(), atol=1e-12 * np.abs(Phi).max())
    # the last forcing enters as kappa * g_{N-1} through the one-step map Phi1
    Phi1 = np.zeros((n, n))
    for col in range(n):
        e = np.zeros(n); e[col] = 1.0
        Phi1[:, col] = heat.heat_steps(e.reshape(X0.shape), zero_g[:1], ALPHA, DT, 1).ravel()
    assert np.allclose(dg[-1].ravel(), DT * (Phi1.T @ c.ravel()), atol=1e-12 * np.abs(Phi1).max())


def test_gradients_with_wall_data_match_central_differences():
    """Run with non-zero Dirichlet data (lifting): dL/dalpha carries the
    alpha-dependence of the lifted right side; all three gradients against
    central differences of the lifted forward run."""
    X0, g, tgt = _problem(3)
    from oracle import transforms as tr
    bc = tr.coeffs2vals(inputs.smooth_coeffs(P, M, N, 1.1, np.random.default_rng(9)))

    def loss(X0_, g_, alpha_):
        XN_ = heat.heat_steps(X0_, g_, alpha_, DT, STEPS, bc=bc)
        return float(np.sum((XN_ - tgt) ** 2))

    XN = heat.heat_steps(X0, g, ALPHA, DT, STEPS, bc=bc)
    dX0, dg, dal = heat.heat_adjoint(X0, g, ALPHA, DT, STEPS, 2.0 * (XN - tgt), bc=bc)
    rng = np.random.default_rng(12)
    h = 1e-3
    d = rng.standard_normal(X0.shape)
    fd = (loss(X0 + h * d, g, ALPHA) - loss(X0 - h * d, g, ALPHA)) / (2 * h)
    assert abs(fd - float(np.sum(dX0 * d))) <= 1e-7 * abs(fd)
    d = rng.standard_normal(g.shape)
    fd = (loss(X0, g + h * d, ALPHA) - loss(X0, g - h * d, ALPHA)) / (2 * h)
    assert abs(fd - float(np.sum(dg * d))) <= 1e-7 * abs(fd)
    h = 1e-4 * ALPHA
    fd = (loss(X0, g, ALPHA + h) - loss(X0, g, ALPHA - h)) / (2 * h)
    assert abs(fd - dal) <= 1e-7 * abs(fd)
    # the wall term matters: dropping it changes dL/dalpha
    _, _, dal0 = heat.heat_adjoint(X0, g, ALPHA, DT, STEPS, 2.0 * (XN - tgt))
    assert abs(dal0 - dal) > 1e-4 * abs(fd)
