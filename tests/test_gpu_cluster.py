"""Cluster mode of the ADI launch (several CTAs of a thread-block cluster per
work item, work arrays in global memory, twisted solves per CTA), against
the FP64 oracle: forced on small grids for every kind of run (Poisson, BDF1
with checkpoints, the BDF2 history ring, non-zero wall data), against the
single-CTA path, at 256^3 on sampled slices, and the bounded
waits' timeout report under a cluster launch."""
import os

import numpy as np
import pytest

from oracle import heat as oheat, transforms as otr
from paper_2206_04827_gb300 import inputs

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

TOL_SOLVE = 1e-12
GOLD256 = os.path.join(os.path.dirname(__file__), 'golden', 'heat256_sampled.npz')


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


@pytest.mark.parametrize('m,n,p', [(12, 11, 4), (33, 33, 16), (40, 37, 8)])
def test_forced_cluster_poisson_and_heat_match_oracle(cyl, m, n, p):
    rng = np.random.default_rng(m * 7 + n)
    F = inputs.smooth_coeffs(p, m, n, 1.2, rng)
    g = inputs.smooth_coeffs(p, m, n, 1.25, rng)
    plan = cyl.Plan(m, n, p, 0.7, 2e-3, 1e-14, poisson=True, heat=True, extra_flags=cyl.FORCE_CLUSTER)
    u = plan.poisson(dev(F), torch.empty(p, m, n, dtype=torch.float64, device='cuda'), cyl.COEFFS)
    plan.sync()
    assert relerr(host(u), oheat.poisson(F)) <= TOL_SOLVE
    steps, every = 5, 2
    T = dev(F)
    ck = torch.zeros(steps // every + 1, p, m, n, dtype=torch.float64, device='cuda')
    plan.heat_step(T, dev(g), steps, ckpt=ck, ckpt_every=every)
    plan.sync()
    _, traj = oheat.heat_steps(F, g, 0.7, 2e-3, steps, return_all=True)
    assert relerr(host(T), traj[-1]) <= TOL_SOLVE
    ckh = host(ck)
    for s in range(steps // every + 1):
        assert relerr(ckh[s], traj[s * every]) <= TOL_SOLVE


def test_forced_cluster_bdf2_and_wall_data_match_oracle(cyl):
    m, n, p = 24, 21, 8
    rng = np.random.default_rng(21)
    X0 = inputs.smooth_coeffs(p, m, n, 1.25, rng)
    g = inputs.smooth_coeffs(p, m, n, 1.25, rng)
    plan = cyl.Plan(m, n, p, 0.5, 5e-3, 1e-14, poisson=False, heat=True, bdf_order=2,
                    extra_flags=cyl.FORCE_CLUSTER)
    H = torch.zeros(2, p, m, n, dtype=torch.float64, device='cuda')
    H[0].copy_(dev(X0))
    plan.heat_step_bdf(H, 1, dev(g), 6)
    plan.sync()
    hist = np.zeros((2, p, m, n))
    hist[0] = X0
    want = oheat.heat_bdf(hist, g, 0.5, 5e-3, 2, 6, nvalid=1)
    assert relerr(host(H), want) <= TOL_SOLVE
    bc = otr.coeffs2vals(inputs.smooth_coeffs(p, m, n, 1.2, rng))
    pw = cyl.Plan(m, n, p, 0.5, 5e-3, 1e-14, poisson=True, heat=True, extra_flags=cyl.FORCE_CLUSTER | cyl.WITH_BC)
    F = inputs.smooth_coeffs(p, m, n, 1.2, rng)
    u = pw.poisson(dev(F), torch.empty(p, m, n, dtype=torch.float64, device='cuda'), cyl.COEFFS, bc=dev(bc))
    pw.sync()
    assert relerr(host(u), oheat.poisson(F, bc=bc)) <= TOL_SOLVE


def test_cluster_equals_single_cta_path(cyl):
    """The same twisted arithmetic split over a cluster of CTAs: agreement
    with the one-CTA-per-item launch to rounding."""
    m = n = p = 64
    rng = np.random.default_rng(4)
    F = dev(inputs.smooth_coeffs(p, m, n, 1.15, rng))
    outs = []
    for flags in (0, cyl.FORCE_CLUSTER):
        plan = cyl.Plan(m, n, p, 0.3, 1e-3, 1e-14, poisson=True, heat=True, extra_flags=flags)
        T = torch.empty_like(F)
        plan.poisson(F, T, cyl.COEFFS)
        plan.heat_step(T, F, 3)
        plan.sync()
        outs.append(host(T))
        plan.close()
    assert relerr(outs[1], outs[0]) <= 1e-13


def test_cluster_256_cubed_sampled_slices_match_oracle(cyl):
    """256^3 in cluster mode (two CTAs per item; one item's iterate exceeds an
    SM's shared memory): 5 BDF1 steps from smooth coefficients, compared on
    sampled slices and coefficients with refined oracle values written by
    tests/golden/make_heat256.py (the plain direct solve itself drifts by
    ~3e-12 over these steps on the k = 0 slice); the default launch
    (single-slice items, twisted solves, iterate in shared memory) and the
    plain one (two-slice items, one-sided sweeps, global work arrays) are held
    to the same values."""
    ref = np.load(GOLD256)
    p = m = n = 256
    rng = inputs.rng_for(int(ref['seed']))
    X0 = inputs.smooth_coeffs(p, m, n, float(ref['decay']), rng)
    g = inputs.smooth_coeffs(p, m, n, float(ref['decay']), rng)
    sl = torch.as_tensor(ref['slices'], device='cuda')
    idx = torch.as_tensor(ref['idx'], device='cuda')
    errs = []
    for flags in (cyl.FORCE_CLUSTER, 0, cyl.PLAIN_SWEEPS):
        plan = cyl.Plan(m, n, p, float(ref['alpha']), float(ref['dt']), 1e-15, poisson=False, heat=True,
                        extra_flags=flags)
        if flags == 0:
            li = plan.launch_info(1)
            assert (li['slices'], li['twist_half'], li['placement']) == (1, 128, 1), li
        T = dev(X0)
        plan.heat_step(T, dev(g), int(ref['steps']))
        plan.sync()
        got = T.index_select(0, sl).index_select(1, idx).index_select(2, idx).cpu().numpy()
        errs.append(relerr(got, ref['heat']))
        plan.close()
    print('256^3 vs refined oracle: cluster %.2e, default %.2e, plain %.2e' % tuple(errs))
    assert max(errs) <= TOL_SOLVE, errs


def test_cluster_bounded_wait_timeout_is_reported(cyl):
    """Under a cluster launch the bounded table waits still run out without
    a fault (no table copy is ever started), every CTA reaches every cluster
    barrier, cyl_sync reports CYL_ETIMEOUT and the context stays usable."""
    p, m, n = 4, 12, 11
    X0 = inputs.smooth_coeffs(p, m, n, 1.3, np.random.default_rng(2))
    bad = cyl.Plan(m, n, p, 0.5, 1e-2, 1e-12, poisson=False, heat=True,
                   extra_flags=cyl.TEST_NO_TMA | cyl.FORCE_CLUSTER)
    T = dev(X0)
    bad.heat_step(T, None, 1)
    with pytest.raises(cyl.CylError) as ei:
        bad.sync()
    assert ei.value.status == cyl.ETIMEOUT
    good = cyl.Plan(m, n, p, 0.5, 1e-2, 1e-14, poisson=False, heat=True, extra_flags=cyl.FORCE_CLUSTER)
    T = dev(X0)
    good.heat_step(T, None, 2)
    good.sync()
    assert relerr(host(T), oheat.heat_steps(X0, np.zeros_like(X0), 0.5, 1e-2, 2)) <= TOL_SOLVE
