"""GPU parity of the BDF2-BDF4 runs (Section 3, BDF 4 and the kappa^(b),
delta^(b) definitions) through the C ABI against the oracle's heat_bdf:
start-up through lower orders, full histories, the history ring's final
order, split runs, boundary data, the scalar recurrence of an eigenmode, and
the multistep adjoint (oracle parity, autograd against central
differences)."""
import numpy as np
import pytest

from oracle import grid, heat as oheat, transforms as otr
from paper_2206_04827_gb300 import inputs

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

TOL_SOLVE = 1e-12


@pytest.fixture(scope='module')
def cyl():
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    from paper_2206_04827_gb300 import cyl as C
    return C


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def relerr(got, want):
    return np.abs(got - want).max() / max(np.abs(want).max(), 1e-300)


def _history(order, nvalid, p, m, n, rng):
    hist = np.zeros((order, p, m, n))
    for i in range(nvalid):
        hist[i] = inputs.smooth_coeffs(p, m, n, 1.25, rng)
    return hist


@pytest.mark.parametrize('order,nvalid,steps', [(2, 1, 5), (3, 1, 6), (4, 1, 7), (4, 2, 3), (4, 4, 6), (3, 3, 1)])
def test_bdf_run_matches_oracle(cyl, order, nvalid, steps):
    p, m, n = 8, 17, 15
    alpha, dt = 0.6, 0.01
    rng = np.random.default_rng(10 * order + nvalid)
    hist = _history(order, nvalid, p, m, n, rng)
    g = np.stack([inputs.smooth_coeffs(p, m, n, 1.25, rng) for _ in range(steps)])
    plan = cyl.Plan(m, n, p, alpha, dt, 1e-14, poisson=False, heat=True, bdf_order=order)
    H = dev(hist)
    plan.heat_step_bdf(H, nvalid, dev(g), steps, g_step_stride=p * m * n)
    want = oheat.heat_bdf(hist, g, alpha, dt, order, steps, nvalid=nvalid)
    got = host(H)
    for i in range(min(order, nvalid + steps)):
        assert relerr(got[i], want[i]) <= TOL_SOLVE, i


def test_split_run_equals_one_run(cyl):
    """3 steps then 4 steps (the second call starting with a full history)
    equal 7 steps in one call, bit for bit (same launches, same arithmetic)."""
    p, m, n, order = 8, 20, 17, 4
    rng = np.random.default_rng(2)
    hist = _history(order, 1, p, m, n, rng)
    g = inputs.smooth_coeffs(p, m, n, 1.25, rng)
    plan = cyl.Plan(m, n, p, 0.5, 0.02, 1e-14, poisson=False, heat=True, bdf_order=order)
    a, b = dev(hist), dev(hist)
    gd = dev(g)
    plan.heat_step_bdf(a, 1, gd, 7)
    plan.heat_step_bdf(b, 1, gd, 3)
    plan.heat_step_bdf(b, 4, gd, 4)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    before = b.clone()
    plan.heat_step_bdf(b, 4, gd, 0)
    assert torch.equal(b, before)


def test_bdf_with_wall_data_matches_oracle(cyl):
    p, m, n, order, steps = 8, 19, 16, 3, 5
    alpha, dt = 0.7, 0.01
    rng = np.random.default_rng(8)
    hist = _history(order, 2, p, m, n, rng)
    g = inputs.smooth_coeffs(p, m, n, 1.25, rng)
    bc = otr.coeffs2vals(inputs.smooth_coeffs(p, m, n, 1.15, rng))
    plan = cyl.Plan(m, n, p, alpha, dt, 1e-14, poisson=False, heat=True, bdf_order=order)
    H = dev(hist)
    plan.heat_step_bdf(H, 2, dev(g), steps, bc=dev(bc))
    want = oheat.heat_bdf(hist, g, alpha, dt, order, steps, nvalid=2, bc=bc)
    got = host(H)
    for i in range(order):
        assert relerr(got[i], want[i]) <= TOL_SOLVE, i


def test_bdf4_at_64_cubed_matches_oracle_on_sampled_slices(cyl):
    p, m, n, order, steps = 64, 64, 64, 4, 8
    alpha, dt = 1.0, 1e-3
    rng = np.random.default_rng(64)
    hist = _history(order, 1, p, m, n, rng)
    g = inputs.smooth_coeffs(p, m, n, 1.25, rng)
    plan = cyl.Plan(m, n, p, alpha, dt, 1e-14, poisson=False, heat=True, bdf_order=order)
    H = dev(hist)
    plan.heat_step_bdf(H, 1, dev(g), steps)
    slices = [0, 1, 2, 17, 18, 40, 63]
    want = oheat.heat_bdf(hist, g, alpha, dt, order, steps, nvalid=1, slices=slices)
    got = host(H)
    for i in range(order):
        assert relerr(got[i][slices], want[i][slices]) <= TOL_SOLVE, i


def test_eigenmode_scalar_recurrence_on_gpu(cyl):
    """A Dirichlet eigenmode under BDF 4 with start-up: the GPU field is the
    scalar BDF recurrence times the mode (independent of the oracle's solver)."""
    p, m, n, order, steps = 8, 33, 33, 4, 9
    alpha, h = 0.8, 0.01
    r, z, th = grid.cheb_points(m), grid.cheb_points(n), grid.theta_points(p)
    E = otr.vals2coeffs(inputs.eigenmode_values(r, z, th, [(2, 1, 1, 1.0)]))
    lam = inputs.eigenvalue(2, 1)
    hist = np.zeros((order, p, m, n))
    hist[0] = E
    plan = cyl.Plan(m, n, p, alpha, h, 1e-14, poisson=False, heat=True, bdf_order=order)
    H = dev(hist)
    plan.heat_step_bdf(H, 1, None, steps)
    amps = [1.0]
    for _ in range(steps):
        b = min(order, len(amps))
        kap, beta = oheat.bdf_coefficients(b)
        nxt = sum(float(beta[i]) * amps[i] for i in range(b)) / (1 + float(kap) * h * alpha * lam)
        amps = [nxt] + amps[:order - 1]
    got = host(H)
    for i in range(order):
        assert np.abs(got[i] - amps[i] * E).max() < 1e-11 * np.abs(E).max(), i


def test_bdf_argument_checks(cyl):
    plan = cyl.Plan(9, 8, 4, 0.5, 0.01, 1e-12, poisson=False, heat=True, bdf_order=3)
    H = torch.zeros(3 * 4 * 9 * 8, dtype=torch.float64, device='cuda')
    for nv in (0, 4):
        with pytest.raises(cyl.CylError) as ei:
            plan.heat_step_bdf(H, nv, None, 1)
        assert ei.value.status == cyl.EINVAL


@pytest.mark.parametrize('order,nvalid,steps,every,varying,wall', [
    (2, 1, 5, 2, True, False), (4, 1, 7, 3, False, False), (4, 4, 6, 4, True, False),
    (3, 2, 5, 5, True, True), (4, 2, 1, 1, False, False)])
def test_bdf_adjoint_matches_oracle(cyl, order, nvalid, steps, every, varying, wall):
    p, m, n = 6, 11, 9
    alpha, dt = 0.6, 0.02
    rng = np.random.default_rng(100 + 10 * order + nvalid + steps)
    hist = _history(order, nvalid, p, m, n, rng)
    g = (np.stack([inputs.smooth_coeffs(p, m, n, 1.3, rng) for _ in range(steps)]) if varying
         else inputs.smooth_coeffs(p, m, n, 1.3, rng))
    lamN = np.stack([inputs.smooth_coeffs(p, m, n, 1.3, rng) for _ in range(order)])
    keep = min(order, nvalid + steps)
    lamN[keep:] = 0.0
    bc = otr.coeffs2vals(inputs.smooth_coeffs(p, m, n, 1.15, rng)) if wall else None
    plan = cyl.Plan(m, n, p, alpha, dt, 1e-14, poisson=False, heat=True, bdf_order=order)
    dh = torch.empty(order, p, m, n, dtype=torch.float64, device='cuda')
    dg = torch.empty(g.shape, dtype=torch.float64, device='cuda')
    dal = torch.zeros(1, dtype=torch.float64, device='cuda')
    plan.heat_adjoint_bdf(dev(hist), nvalid, dev(g), steps, dev(lamN), dh, dg, dal,
                          g_step_stride=(p * m * n if varying else 0), ckpt_every=every,
                          bc=dev(bc) if wall else None)
    w0, wg, wa = oheat.heat_bdf_adjoint(hist, g, alpha, dt, order, steps, lamN, nvalid=nvalid, bc=bc)
    got = host(dh)
    assert relerr(got[:nvalid], w0[:nvalid]) <= TOL_SOLVE
    assert np.all(got[nvalid:] == 0.0)
    assert relerr(host(dg), wg) <= TOL_SOLVE
    assert abs(host(dal)[0] - wa) <= 1e-10 * abs(wa)
    # without dL/dalpha: same history and forcing gradients, no recomputation
    dh2 = torch.empty_like(dh)
    plan.heat_adjoint_bdf(None, nvalid, dev(g), steps, dev(lamN), dh2, None, None,
                          g_step_stride=(p * m * n if varying else 0))
    assert relerr(host(dh2)[:nvalid], w0[:nvalid]) <= TOL_SOLVE


def test_bdf_autograd_alpha_against_central_differences(cyl):
    """torch.autograd through a BDF 4 run with start-up at 33^3 x 24 steps:
    d/dalpha of a quadratic loss of the final history against central
    differences of the GPU forward run."""
    from paper_2206_04827_gb300.autograd import heat_bdf
    p, m, n, order, steps = 16, 33, 33, 4, 24
    rng = np.random.default_rng(77)
    H0 = torch.zeros(order, p, m, n, dtype=torch.float64, device='cuda')
    H0[0] = dev(inputs.smooth_coeffs(p, m, n, 1.25, rng))
    g = dev(inputs.smooth_coeffs(p, m, n, 1.25, rng))
    tgt = dev(np.stack([inputs.smooth_coeffs(p, m, n, 1.25, rng) for _ in range(order)]))
    dt, alpha0 = 2e-3, 0.7
    a = torch.tensor(alpha0, dtype=torch.float64, device='cuda', requires_grad=True)
    Hr = H0.clone().requires_grad_(True)
    loss = ((heat_bdf(Hr, g, a, dt, order, steps, nvalid=1, ckpt_every=5) - tgt) ** 2).sum()
    loss.backward()

    def L(H, al):
        with torch.no_grad():
            return float(((heat_bdf(H, g, al, dt, order, steps, nvalid=1) - tgt) ** 2).sum())

    h = 1e-4 * alpha0
    fd = (L(H0, alpha0 + h) - L(H0, alpha0 - h)) / (2 * h)
    assert abs(float(a.grad) - fd) <= 1e-7 * abs(fd)
    # the initial-state gradient along a random direction
    d = torch.zeros_like(H0)
    d[0] = dev(inputs.smooth_coeffs(p, m, n, 1.25, rng))
    eps = 1e-3
    fd = (L(H0 + eps * d, alpha0) - L(H0 - eps * d, alpha0)) / (2 * eps)
    assert abs(float((Hr.grad * d).sum()) - fd) <= 1e-7 * abs(fd)
