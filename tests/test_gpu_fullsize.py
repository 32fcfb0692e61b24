"""Parity at the workloads' full sizes, in the launch configurations the
benchmark times, against the FP64 oracle on the same seeded inputs:

* value <-> coefficient transforms (Section 2) on the 128^3 grid and on
  512-point axes, element by element, <= 1e-13 relative max-norm;
* the 256-problem batch (n_r, n_z ~ U{32..256}, n_theta in {32, 64, 128},
  alpha ~ U[0.01, 1], dt 1e-3, the benchmark's seed) in the configuration
  the autotuner picks, on sampled slices of sampled problems (the three
  largest and three drawn at random), <= 1e-12;
* the 128^3 adjoint (alpha 0.5, dt 1e-3, 200 BDF1 steps, checkpoint every
  20, space-time forcing) element by element on sampled slices and time
  levels: dL/dT0 and dL/dg against the oracle's chain-rule adjoint,
  <= 1e-7 (the gradient tolerance), and the final state <= 1e-12.

Slices (wavenumbers) are independent, so the oracle solves only the sampled
slices of a full-size problem."""
import numpy as np
import pytest

from oracle import heat as oheat, transforms as otr
from paper_2206_04827_gb300 import inputs

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

TOL_XFORM = 1e-13
TOL_SOLVE = 1e-12
TOL_GRAD = 1e-7


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


@pytest.mark.parametrize('m,n,p', [(128, 128, 128), (512, 33, 8), (33, 512, 8), (9, 17, 512)])
def test_transforms_full_size_match_oracle(cyl, m, n, p):
    rng = np.random.default_rng(500 + m + 3 * n + 7 * p)
    vals = rng.standard_normal((p, m, n))
    plan = cyl.Plan(m, n, p)
    c = host(plan.vals2coeffs(dev(vals), torch.empty(p, m, n, dtype=torch.float64, device='cuda')))
    assert relerr(c, otr.vals2coeffs(vals)) <= TOL_XFORM
    H = inputs.smooth_coeffs(p, m, n, 1.02, rng) + 1e-3 * rng.standard_normal((p, m, n))
    v = host(plan.coeffs2vals(dev(H), torch.empty(p, m, n, dtype=torch.float64, device='cuda')))
    assert relerr(v, otr.coeffs2vals(H)) <= TOL_XFORM
    plan.close()


def _c3_batch(k=256):
    """The 256-problem heat workload's problems and forcing (seed 1003, the
    draw order of the benchmark)."""
    rng = inputs.rng_for(1003)
    n_r = rng.integers(32, 257, size=k)
    n_z = rng.integers(32, 257, size=k)
    n_t = rng.choice([32, 64, 128], size=k)
    alpha = rng.uniform(0.01, 1.0, size=k)
    return rng, n_r, n_z, n_t, alpha


def test_batch_256_problems_autotuned_match_oracle(cyl):
    rng, n_r, n_z, n_t, alpha = _c3_batch()
    dt, steps = 1e-3, 10
    bp = cyl.BatchPlan(n_r, n_z, n_t, alpha, dt, 1e-14)
    gs = [inputs.smooth_coeffs(p, m, n, 1.25, rng) for p, m, n in bp.shapes]
    g = torch.cat([dev(x).reshape(-1) for x in gs])
    T = torch.zeros_like(g)
    bp.autotune(T, g, 1)
    thr, G, counts = bp.config()
    assert sum(counts) > 0
    T.zero_()
    bp.heat_step(T, g, steps)
    bp.sync()
    # the three problems with the largest min(n_r, n_z), three more at random
    big = list(np.argsort(-np.minimum(n_r, n_z))[:3])
    assert all(min(n_r[i], n_z[i]) >= 200 for i in big)
    rest = [i for i in np.random.default_rng(5).permutation(len(n_r)) if i not in big][:3]
    for i in big + rest:
        p, m, n = bp.shapes[i]
        sl = [0, 1, p // 2, p - 2]
        got = host(bp.view(T, i))
        want = oheat.heat_steps(np.zeros((p, m, n)), gs[i], float(alpha[i]), dt, steps, slices=sl)
        scale = np.abs(want[sl]).max()
        err = max(np.abs(got[s] - want[s]).max() for s in sl) / scale
        assert err <= TOL_SOLVE, (i, (p, m, n), err)


def test_adjoint_128_200_steps_sampled_slices_match_oracle(cyl):
    p = m = n = 128
    steps, every = 200, 20
    alpha, dt = 0.5, 1e-3
    N = p * m * n
    rng = inputs.rng_for(1004)
    r = np.cos((m - 1 - np.arange(m)) * np.pi / (m - 1))
    th = (2 * np.arange(p) - p) * np.pi / p
    plan = cyl.Plan(m, n, p, alpha, dt, 1e-14, poisson=False, heat=True)
    T0 = plan.vals2coeffs(dev(inputs.eigenmode_values(r, r, th, inputs.eigenmode_list(8, rng))),
                          torch.empty(p, m, n, dtype=torch.float64, device='cuda'))
    sl = [0, 1, 64, 126]
    levels = [0, 1, 57, 100, 198, 199]
    # forcing on the device, and on the host only where the oracle reads it
    g = torch.empty((steps, p, m, n), dtype=torch.float64, device='cuda')
    g_host = np.zeros((steps, p, m, n))
    for s in range(steps):
        x = inputs.smooth_coeffs(p, m, n, 1.25, rng)
        g[s].copy_(torch.as_tensor(x))
        g_host[s, sl] = x[sl]
    tgt = dev(inputs.smooth_coeffs(p, m, n, 1.25, rng))
    w = torch.full((p, 1, 1), 2.0, dtype=torch.float64, device='cuda')
    w[0] = w[p - 1] = 1.0
    # the benchmark's launch sequence: forward run writing checkpoints, adjoint reading them
    T = T0.clone()
    ck = torch.empty((steps // every + 1) * N, dtype=torch.float64, device='cuda')
    plan.heat_step(T, g, steps, g_step_stride=N, ckpt=ck, ckpt_every=every)
    lamN = 2.0 * w * (T - tgt)
    dT0 = torch.empty_like(T0)
    dg = torch.empty_like(g)
    dal = torch.zeros(1, dtype=torch.float64, device='cuda')
    plan.heat_adjoint(T0, g, steps, lamN, dT0, dg, dal, g_step_stride=N, ckpt_every=every, ckpt=ck)
    plan.sync()
    X0h = np.zeros((p, m, n))
    X0h[sl] = host(T0)[sl]
    lamh = np.zeros((p, m, n))
    lamh[sl] = host(lamN)[sl]
    XN = oheat.heat_steps(X0h, g_host, alpha, dt, steps, slices=sl)
    Th = host(T)
    assert max(np.abs(Th[s] - XN[s]).max() for s in sl) / np.abs(XN[sl]).max() <= TOL_SOLVE
    w0, wg, _ = oheat.heat_adjoint(X0h, g_host, alpha, dt, steps, lamh, slices=sl)
    d0 = host(dT0)
    assert max(np.abs(d0[s] - w0[s]).max() for s in sl) / np.abs(w0[sl]).max() <= TOL_GRAD
    dgl = dg[levels].cpu().numpy()
    scale = np.abs(wg[levels][:, sl]).max()
    err = max(np.abs(dgl[q, s] - wg[lv, s]).max() for q, lv in enumerate(levels) for s in sl) / scale
    assert err <= TOL_GRAD
