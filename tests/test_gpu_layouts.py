"""Launch layouts of the ADI kernels beyond shared memory, against the FP64
oracle: single-slice items with twisted solves on two threads per chain
(grids whose two-slice work arrays leave shared memory; here 300 x 300,
class size 149, 2 x 160 threads, work arrays in global memory) for Poisson,
BDF1 with checkpoints and the adjoint with its alpha gradient; and one-sided
sweeps with more chains than threads (a 520-point vertical axis: 518 radial
chains on 512 threads)."""
import numpy as np
import pytest

from oracle import heat as oheat
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


def test_twisted_single_slice_items_match_oracle(cyl):
    p, m, n = 4, 300, 300
    rng = np.random.default_rng(300)
    F = inputs.smooth_coeffs(p, m, n, 1.15, rng)
    g = inputs.smooth_coeffs(p, m, n, 1.15, rng)
    alpha, dt, steps, every = 0.4, 1e-3, 3, 2
    plan = cyl.Plan(m, n, p, alpha, dt, 1e-15, poisson=True, heat=True)
    for which in (0, 1):
        li = plan.launch_info(which)
        assert (li['slices'], li['twist_half'], li['threads'], li['placement']) == (1, 160, 320, 0), li
    u = plan.poisson(dev(F), torch.empty(p, m, n, dtype=torch.float64, device='cuda'), cyl.COEFFS)
    plan.sync()
    assert relerr(host(u), oheat.poisson(F)) <= TOL_SOLVE
    T = dev(F)
    ck = torch.zeros(steps // every + 1, p, m, n, dtype=torch.float64, device='cuda')
    plan.heat_step(T, dev(g), steps, ckpt=ck, ckpt_every=every)
    plan.sync()
    _, traj = oheat.heat_steps(F, g, alpha, dt, steps, return_all=True)
    assert relerr(host(T), traj[-1]) <= TOL_SOLVE
    ckh = host(ck)
    for s in range(steps // every + 1):
        assert relerr(ckh[s], traj[s * every]) <= TOL_SOLVE


def test_twisted_single_slice_adjoint_matches_oracle(cyl):
    """The adjoint kernel on the same layout (twisted records of the flipped
    transposes, 2 x 160 threads), gradients in T0, a space-time g and alpha."""
    p, m, n, steps = 4, 300, 300, 3
    alpha, dt = 0.4, 1e-3
    rng = np.random.default_rng(301)
    X0 = inputs.smooth_coeffs(p, m, n, 1.15, rng)
    g = np.stack([inputs.smooth_coeffs(p, m, n, 1.15, rng) for _ in range(steps)])
    lamN = inputs.smooth_coeffs(p, m, n, 1.15, rng)
    plan = cyl.Plan(m, n, p, alpha, dt, 1e-15, poisson=False, heat=True)
    assert plan.launch_info(1)['threads'] == 320
    dT0 = torch.empty(p, m, n, dtype=torch.float64, device='cuda')
    dg = torch.empty(g.shape, dtype=torch.float64, device='cuda')
    dal = torch.zeros(1, dtype=torch.float64, device='cuda')
    plan.heat_adjoint(dev(X0), dev(g), steps, dev(lamN), dT0, dg, dal, g_step_stride=p * m * n, ckpt_every=2)
    plan.sync()
    w0, wg, wa = oheat.heat_adjoint(X0, g, alpha, dt, steps, lamN)
    assert relerr(host(dT0), w0) <= 1e-11
    assert relerr(host(dg), wg) <= 1e-11
    assert abs(host(dal)[0] - wa) <= 1e-9 * abs(wa)


def test_more_chains_than_threads_match_oracle(cyl):
    """n_z = 520: the radial sweeps of a two-slice item have 2 x 259 chains,
    run by 512 threads (the first six take a second chain)."""
    p, m, n = 4, 8, 520
    rng = np.random.default_rng(520)
    F = inputs.smooth_coeffs(p, m, n, 1.05, rng)
    plan = cyl.Plan(m, n, p, 0.5, 1e-3, 1e-15, poisson=True, heat=True)
    li = plan.launch_info(0)
    assert li['threads'] == 512 and li['twist_half'] == 0 and li['slices'] == 2, li
    u = plan.poisson(dev(F), torch.empty(p, m, n, dtype=torch.float64, device='cuda'), cyl.COEFFS)
    plan.sync()
    assert relerr(host(u), oheat.poisson(F)) <= TOL_SOLVE
    T = dev(F)
    plan.heat_step(T, dev(F), 2)
    plan.sync()
    assert relerr(host(T), oheat.heat_steps(F, F, 0.5, 1e-3, 2)) <= TOL_SOLVE
