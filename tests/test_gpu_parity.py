"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  Bars (relative max-norm, max|gpu - oracle| / max|oracle|):
transforms <= 1e-13, solves <= 1e-12 on the coefficients."""
import numpy as np
import pytest

from oracle import grid, heat as oheat, transforms as otr
from paper_2206_04827_gb300 import inputs

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

TOL_XFORM = 1e-13
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


SIZES = [(4, 4, 2), (5, 6, 4), (9, 8, 6), (16, 17, 8), (33, 33, 32), (40, 37, 16)]


@pytest.mark.parametrize('m,n,p', SIZES)
def test_transforms_match_oracle(cyl, m, n, p):
    rng = np.random.default_rng(100 + m + n + p)
    vals = rng.standard_normal((p, m, n))
    plan = cyl.Plan(m, n, p)
    c = plan.vals2coeffs(dev(vals), torch.empty(p, m, n, dtype=torch.float64, device='cuda'))
    want = otr.vals2coeffs(vals)
    assert relerr(host(c), want) <= TOL_XFORM
    H = rng.standard_normal((p, m, n))
    v = plan.coeffs2vals(dev(H), torch.empty(p, m, n, dtype=torch.float64, device='cuda'))
    assert relerr(host(v), otr.coeffs2vals(H)) <= TOL_XFORM
    # in-place use
    t = dev(vals)
    plan.vals2coeffs(t, t)
    assert relerr(host(t), want) <= TOL_XFORM


@pytest.mark.parametrize('m,n,p', SIZES[1:])
def test_poisson_coeffs_match_oracle(cyl, m, n, p):
    F = inputs.smooth_coeffs(p, m, n, 1.2, np.random.default_rng(7 * m + n))
    plan = cyl.Plan(m, n, p, adi_tol=1e-14)
    u = plan.poisson(dev(F), torch.empty(p, m, n, dtype=torch.float64, device='cuda'), cyl.COEFFS)
    plan.sync()
    assert relerr(host(u), oheat.poisson(F)) <= TOL_SOLVE


def test_poisson_manufactured_values_33(cyl):
    """The 33 x 33 x 32 manufactured problem, values in, values out."""
    p, m, n = 32, 33, 33
    r, z, th = grid.cheb_points(m), grid.cheb_points(n), grid.theta_points(p)
    f = inputs.manufactured_f(r, z, th)
    plan = cyl.Plan(m, n, p, adi_tol=1e-13)
    fu = dev(f)
    u = host(plan.poisson(fu, fu, cyl.VALUES))        # aliasing in/out is allowed
    ref_c = oheat.poisson(otr.vals2coeffs(f))
    assert relerr(u, otr.coeffs2vals(ref_c)) <= TOL_SOLVE
    assert relerr(u, inputs.manufactured_u(r, z, th)) <= 1e-11


def test_poisson_both_parities_nonphysical_input(cyl):
    p, m, n = 8, 14, 11
    F = np.random.default_rng(3).standard_normal((p, m, n))
    ii, jj = np.meshgrid(np.arange(m), np.arange(n), indexing='ij')
    F *= 1.3 ** (-(ii + jj))[None]
    plan = cyl.Plan(m, n, p, adi_tol=1e-14, both_parities=True)
    u = plan.poisson(dev(F), torch.empty(p, m, n, dtype=torch.float64, device='cuda'), cyl.COEFFS)
    assert relerr(host(u), oheat.poisson(F)) <= TOL_SOLVE


def test_global_work_arrays_equal_shared(cyl):
    p, m, n = 8, 20, 19
    F = inputs.smooth_coeffs(p, m, n, 1.2, np.random.default_rng(9))
    a = cyl.Plan(m, n, p, adi_tol=1e-14)
    b = cyl.Plan(m, n, p, adi_tol=1e-14, force_global=True)
    ua = host(a.poisson(dev(F), torch.empty(p, m, n, dtype=torch.float64, device='cuda'), cyl.COEFFS))
    ub = host(b.poisson(dev(F), torch.empty(p, m, n, dtype=torch.float64, device='cuda'), cyl.COEFFS))
    assert np.array_equal(ua, ub)


@pytest.mark.parametrize('m,n,p,steps', [(9, 8, 6, 3), (24, 21, 8, 5), (33, 33, 16, 4)])
def test_heat_steps_match_oracle(cyl, m, n, p, steps):
    rng = np.random.default_rng(m * 31 + steps)
    X0 = inputs.smooth_coeffs(p, m, n, 1.25, rng)
    g = inputs.smooth_coeffs(p, m, n, 1.25, rng)
    alpha, dt = 0.8, 2e-3
    plan = cyl.Plan(m, n, p, alpha, dt, 1e-14, poisson=False, heat=True)
    T = dev(X0)
    plan.heat_step(T, dev(g), steps)
    plan.sync()
    assert relerr(host(T), oheat.heat_steps(X0, g, alpha, dt, steps)) <= TOL_SOLVE


def test_heat_time_varying_forcing_and_checkpoints(cyl):
    p, m, n, steps, every = 8, 17, 15, 6, 2
    rng = np.random.default_rng(12)
    X0 = inputs.smooth_coeffs(p, m, n, 1.25, rng)
    g = np.stack([inputs.smooth_coeffs(p, m, n, 1.25, rng) for _ in range(steps)])
    alpha, dt = 0.5, 1e-2
    plan = cyl.Plan(m, n, p, alpha, dt, 1e-14, poisson=False, heat=True)
    T = dev(X0)
    ck = torch.zeros(steps // every + 1, p, m, n, dtype=torch.float64, device='cuda')
    plan.heat_step(T, dev(g), steps, g_step_stride=p * m * n, ckpt=ck, ckpt_every=every)
    _, traj = oheat.heat_steps(X0, g, alpha, dt, steps, return_all=True)
    assert relerr(host(T), traj[-1]) <= TOL_SOLVE
    ckh = host(ck)
    for s in range(steps // every + 1):
        assert relerr(ckh[s], traj[s * every]) <= TOL_SOLVE


def test_heat_eigenmode_decay_128(cyl):
    """Full 128^3, 100 steps, alpha = 1, dt = 1e-3: T0 = 8 Bessel x sine
    eigenmodes; each mode decays by exactly (1 + alpha dt lambda)^-100 under
    BDF1 (spatial error is spectrally small), checked on the whole field."""
    p = m = n = 128
    rng = inputs.rng_for(1001)
    modes = inputs.eigenmode_list(8, rng)
    r, z, th = grid.cheb_points(m), grid.cheb_points(n), grid.theta_points(p)
    plan = cyl.Plan(m, n, p, 1.0, 1e-3, 1e-14, poisson=False, heat=True)
    T = plan.vals2coeffs(dev(inputs.eigenmode_values(r, z, th, modes)),
                         torch.empty(p, m, n, dtype=torch.float64, device='cuda'))
    plan.heat_step(T, None, 100)
    got = host(T)
    decayed = [(mu, nu, t, a * (1 + 1e-3 * inputs.eigenvalue(mu, nu)) ** -100) for mu, nu, t, a in modes]
    want = otr.vals2coeffs(inputs.eigenmode_values(r, z, th, decayed))
    assert relerr(got, want) <= 1e-11


def test_heat_128_sampled_slices_match_oracle(cyl):
    """Full 128^3 heat run (alpha 1, dt 1e-3, 20 steps, smooth forcing) compared
    with the oracle on sampled slices (the oracle steps only those slices;
    slices are independent)."""
    p = m = n = 128
    rng = inputs.rng_for(1001)
    X0 = inputs.smooth_coeffs(p, m, n, 1.25, rng)
    g = inputs.smooth_coeffs(p, m, n, 1.25, rng)
    steps = 20
    plan = cyl.Plan(m, n, p, 1.0, 1e-3, 1e-14, poisson=False, heat=True)
    T = dev(X0)
    plan.heat_step(T, dev(g), steps)
    got = host(T)
    sl = [0, 1, 2, 5, 64, 127]
    want = oheat.heat_steps(X0, g, 1.0, 1e-3, steps, slices=sl)
    scale = np.abs(want[sl]).max()
    for s in sl:
        assert np.abs(got[s] - want[s]).max() / scale <= TOL_SOLVE, s


def test_bounded_wait_timeout_is_reported(cyl):
    """Failure detection without a GPU fault: under CYL_TEST_NO_TMA no table
    copy is ever started, every bounded wait runs out, cyl_sync reports
    CYL_ETIMEOUT, and the context stays usable afterwards."""
    p, m, n = 4, 9, 8
    X0 = inputs.smooth_coeffs(p, m, n, 1.3, np.random.default_rng(1))
    bad = cyl.Plan(m, n, p, 0.5, 1e-2, 1e-12, poisson=False, heat=True, extra_flags=cyl.TEST_NO_TMA)
    T = dev(X0)
    bad.heat_step(T, None, 1)
    with pytest.raises(cyl.CylError) as ei:
        bad.sync()
    assert ei.value.status == cyl.ETIMEOUT
    bad.sync()                                        # the flag was cleared
    good = cyl.Plan(m, n, p, 0.5, 1e-2, 1e-14, poisson=False, heat=True)
    T = dev(X0)
    good.heat_step(T, None, 2)
    good.sync()
    assert relerr(host(T), oheat.heat_steps(X0, np.zeros_like(X0), 0.5, 1e-2, 2)) <= TOL_SOLVE
