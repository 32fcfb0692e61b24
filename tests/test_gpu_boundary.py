"""GPU parity of non-zero Dirichlet data (lifting) through the C ABI against
the oracle's lifted solves: Poisson in both spaces, BDF1 runs, both parity
blocks with rough data, the adjoint of the lifted run, a harmonic function
recovered from its wall values, and graph capture of a plan made with
CYL_WITH_BC."""
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


def _wall(p, m, n, seed, decay=1.15):
    """Grid values of a smooth field on the doubled grid (its boundary nodes
    are the data)."""
    return otr.coeffs2vals(inputs.smooth_coeffs(p, m, n, decay, np.random.default_rng(seed)))


@pytest.mark.parametrize('m,n,p', [(9, 8, 6), (33, 29, 16), (40, 37, 16)])
def test_poisson_with_wall_data_coeffs(cyl, m, n, p):
    F = inputs.smooth_coeffs(p, m, n, 1.2, np.random.default_rng(m + 3 * n))
    bc = _wall(p, m, n, 5 + m)
    plan = cyl.Plan(m, n, p)
    u = plan.poisson(dev(F), torch.empty(p, m, n, dtype=torch.float64, device='cuda'), cyl.COEFFS, bc=dev(bc))
    assert relerr(host(u), oheat.poisson(F, bc=bc)) <= TOL_SOLVE


def test_poisson_with_wall_data_values_in_place(cyl):
    p, m, n = 16, 24, 21
    f = otr.coeffs2vals(inputs.smooth_coeffs(p, m, n, 1.2, np.random.default_rng(1)))
    bc = _wall(p, m, n, 2)
    plan = cyl.Plan(m, n, p)
    fu = dev(f)
    u = host(plan.poisson(fu, fu, cyl.VALUES, bc=dev(bc)))
    want = otr.coeffs2vals(oheat.poisson(otr.vals2coeffs(f), bc=bc))
    assert relerr(u, want) <= TOL_SOLVE
    # the solution meets the data on the four faces
    for sl in (np.s_[:, 0, :], np.s_[:, -1, :], np.s_[:, :, 0], np.s_[:, :, -1]):
        assert np.abs(u[sl] - bc[sl]).max() <= 1e-11 * np.abs(bc).max()


def test_harmonic_function_from_wall_values(cyl):
    """exp(z) cos(x) is harmonic: f = 0 and its wall values alone give it back
    to spectral accuracy (independent of the oracle)."""
    p, m, n = 24, 25, 25
    TH, RR, ZZ = np.meshgrid(grid.theta_points(p), grid.cheb_points(m), grid.cheb_points(n), indexing='ij')
    u = np.exp(ZZ) * np.cos(RR * np.cos(TH))
    plan = cyl.Plan(m, n, p)
    got = host(plan.poisson(dev(np.zeros_like(u)), torch.empty(p, m, n, dtype=torch.float64, device='cuda'),
                            cyl.VALUES, bc=dev(u)))
    assert np.abs(got - u).max() < 1e-11


@pytest.mark.parametrize('m,n,p,steps', [(17, 15, 8, 4), (33, 33, 32, 6)])
def test_heat_with_wall_data_matches_oracle(cyl, m, n, p, steps):
    rng = np.random.default_rng(40 + m)
    alpha, dt = 0.45, 0.01
    X0 = inputs.smooth_coeffs(p, m, n, 1.25, rng)
    g = np.stack([inputs.smooth_coeffs(p, m, n, 1.25, rng) for _ in range(steps)])
    bc = _wall(p, m, n, 7 + m)
    plan = cyl.Plan(m, n, p, alpha, dt, 1e-14, poisson=False, heat=True)
    T = dev(X0)
    ck = torch.empty((steps // 2 + 1) * p * m * n, dtype=torch.float64, device='cuda')
    plan.heat_step(T, dev(g), steps, g_step_stride=p * m * n, ckpt=ck, ckpt_every=2, bc=dev(bc))
    traj = oheat.heat_steps(X0, g, alpha, dt, steps, return_all=True, bc=bc)[1]
    assert relerr(host(T), traj[steps]) <= TOL_SOLVE
    cks = host(ck).reshape(-1, p, m, n)
    for i in range(cks.shape[0]):
        assert relerr(cks[i], traj[2 * i]) <= TOL_SOLVE


def test_both_parities_with_rough_data(cyl):
    """Random wall data (not a field on the doubled grid): both radial parity
    blocks are solved, so the result is still the oracle's."""
    p, m, n = 8, 14, 11
    rng = np.random.default_rng(77)
    F = rng.standard_normal((p, m, n))
    bc = rng.standard_normal((p, m, n))
    plan = cyl.Plan(m, n, p, both_parities=True)
    u = plan.poisson(dev(F), torch.empty(p, m, n, dtype=torch.float64, device='cuda'), cyl.COEFFS, bc=dev(bc))
    assert relerr(host(u), oheat.poisson(F, bc=bc)) <= 1e-11


def test_zero_data_equals_no_data(cyl):
    p, m, n = 8, 17, 13
    F = inputs.smooth_coeffs(p, m, n, 1.2, np.random.default_rng(4))
    plan = cyl.Plan(m, n, p)
    a = host(plan.poisson(dev(F), torch.empty(p, m, n, dtype=torch.float64, device='cuda'), cyl.COEFFS))
    b = host(plan.poisson(dev(F), torch.empty(p, m, n, dtype=torch.float64, device='cuda'), cyl.COEFFS,
                          bc=torch.zeros(p, m, n, dtype=torch.float64, device='cuda')))
    assert np.abs(a - b).max() <= 1e-15 * np.abs(a).max()


def test_adjoint_of_lifted_run_matches_oracle(cyl):
    p, m, n, steps = 6, 11, 9, 5
    alpha, dt = 0.6, 0.02
    rng = np.random.default_rng(31)
    X0 = inputs.smooth_coeffs(p, m, n, 1.3, rng)
    g = np.stack([inputs.smooth_coeffs(p, m, n, 1.3, rng) for _ in range(steps)])
    lamN = inputs.smooth_coeffs(p, m, n, 1.3, rng)
    bc = _wall(p, m, n, 8)
    plan = cyl.Plan(m, n, p, alpha, dt, 1e-14, poisson=False, heat=True)
    dT0 = torch.empty(p, m, n, dtype=torch.float64, device='cuda')
    dg = torch.empty(steps, p, m, n, dtype=torch.float64, device='cuda')
    dal = torch.zeros(1, dtype=torch.float64, device='cuda')
    plan.heat_adjoint(dev(X0), dev(g), steps, dev(lamN), dT0, dg, dal, g_step_stride=p * m * n,
                      ckpt_every=2, bc=dev(bc))
    w0, wg, wa = oheat.heat_adjoint(X0, g, alpha, dt, steps, lamN, bc=bc)
    assert relerr(host(dT0), w0) <= TOL_SOLVE
    assert relerr(host(dg), wg) <= TOL_SOLVE
    assert abs(host(dal)[0] - wa) <= 1e-10 * abs(wa)


def test_autograd_alpha_gradient_with_wall_data(cyl):
    """torch.autograd through the lifted run: d/dalpha of a quadratic loss
    against central differences of the GPU forward run."""
    from paper_2206_04827_gb300.autograd import heat
    p, m, n, steps = 8, 17, 15, 6
    rng = np.random.default_rng(55)
    X0 = dev(inputs.smooth_coeffs(p, m, n, 1.25, rng))
    g = dev(inputs.smooth_coeffs(p, m, n, 1.25, rng))
    tgt = dev(inputs.smooth_coeffs(p, m, n, 1.25, rng))
    bc = dev(_wall(p, m, n, 9))
    dt, alpha0 = 0.01, 0.5
    a = torch.tensor(alpha0, dtype=torch.float64, device='cuda', requires_grad=True)
    loss = ((heat(X0, g, a, dt, steps, ckpt_every=3, bc=bc) - tgt) ** 2).sum()
    loss.backward()

    def L(al):
        with torch.no_grad():
            return float(((heat(X0, g, al, dt, steps, bc=bc) - tgt) ** 2).sum())

    h = 1e-4 * alpha0
    fd = (L(alpha0 + h) - L(alpha0 - h)) / (2 * h)
    assert abs(float(a.grad) - fd) <= 1e-7 * abs(fd)


def test_graph_capture_with_bc_plan(cyl):
    """A plan made with CYL_WITH_BC owns its lifting arrays, so a lifted run
    can be captured in a CUDA graph and replayed."""
    p, m, n, steps = 8, 17, 15, 3
    rng = np.random.default_rng(66)
    X0 = inputs.smooth_coeffs(p, m, n, 1.25, rng)
    g = inputs.smooth_coeffs(p, m, n, 1.25, rng)
    bc = _wall(p, m, n, 10)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan = cyl.Plan(m, n, p, 0.4, 0.01, 1e-14, poisson=False, heat=True, stream=s.cuda_stream,
                        extra_flags=cyl.WITH_BC)
        T, gd, bd = dev(X0), dev(g), dev(bc)
        plan.heat_step(T, gd, steps, bc=bd)          # warm-up outside capture
        s.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            plan.heat_step(T, gd, steps, bc=bd)
        T.copy_(dev(X0))
        graph.replay()
        s.synchronize()
    want = oheat.heat_steps(X0, g, 0.4, 0.01, steps, bc=bc)
    assert relerr(host(T), want) <= TOL_SOLVE
