"""GPU adjoint (cyl_heat_adjoint) against the oracle's chain-rule adjoint, the
transpose identity of the GPU's own forward map, and central finite
differences of the GPU forward; plus the torch.autograd wrapper."""
import numpy as np
import pytest

from oracle import heat as oheat, transforms as otr
from paper_2206_04827_gb300 import inputs

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-7       # gradient bar (finite differences, dense adjoint)


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


def rel(got, want):
    return np.abs(np.asarray(got) - np.asarray(want)).max() / max(np.abs(want).max(), 1e-300)


def _problem(p, m, n, steps, seed, varying=True):
    rng = np.random.default_rng(seed)
    X0 = inputs.smooth_coeffs(p, m, n, 1.3, rng)
    if varying:
        g = np.stack([inputs.smooth_coeffs(p, m, n, 1.3, rng) for _ in range(steps)])
    else:
        g = inputs.smooth_coeffs(p, m, n, 1.3, rng)
    lamN = inputs.smooth_coeffs(p, m, n, 1.3, rng)
    return X0, g, lamN


@pytest.mark.parametrize('varying,every', [(True, 1), (True, 2), (False, 3), (False, 10)])
def test_adjoint_matches_oracle(cyl, varying, every):
    p, m, n, steps = 6, 11, 9, 5
    alpha, dt = 0.6, 0.01
    X0, g, lamN = _problem(p, m, n, steps, 21 + every, varying)
    plan = cyl.Plan(m, n, p, alpha, dt, 1e-14, poisson=False, heat=True)
    dT0 = torch.empty(p, m, n, dtype=torch.float64, device='cuda')
    dg = torch.empty(g.shape, dtype=torch.float64, device='cuda')
    dal = torch.zeros(1, dtype=torch.float64, device='cuda')
    plan.heat_adjoint(dev(X0), dev(g), steps, dev(lamN), dT0, dg, dal,
                      g_step_stride=p * m * n if varying else 0, ckpt_every=every)
    plan.sync()
    w0, wg, wa = oheat.heat_adjoint(X0, g, alpha, dt, steps, lamN)
    assert rel(host(dT0), w0) <= 1e-11
    assert rel(host(dg), wg) <= 1e-11
    assert abs(host(dal)[0] - wa) <= 1e-9 * abs(wa)


def test_adjoint_without_alpha_needs_no_workspace(cyl):
    p, m, n, steps = 4, 10, 10, 4
    X0, g, lamN = _problem(p, m, n, steps, 5, varying=False)
    plan = cyl.Plan(m, n, p, 0.3, 0.02, 1e-14, poisson=False, heat=True)
    assert plan.adjoint_workspace_bytes(steps, 2, False) == 0
    a = torch.empty(p, m, n, dtype=torch.float64, device='cuda')
    plan.heat_adjoint(None, dev(g), steps, dev(lamN), a)
    w0, _, _ = oheat.heat_adjoint(X0, g, 0.3, 0.02, steps, lamN)
    assert rel(host(a), w0) <= 1e-11


def test_transpose_identity_of_gpu_maps(cyl):
    """<c, Phi v> = <Phi^T c, v> with Phi the GPU forward map (g = 0) and
    Phi^T the GPU adjoint, at 33 x 33 x 32 over 10 steps."""
    m = n = 33
    p = 32
    steps = 10
    rng = np.random.default_rng(3)
    v = inputs.smooth_coeffs(p, m, n, 1.2, rng)
    c = inputs.smooth_coeffs(p, m, n, 1.2, rng)
    plan = cyl.Plan(m, n, p, 1.0, 1e-3, 1e-14, poisson=False, heat=True)
    Tv = dev(v)
    plan.heat_step(Tv, None, steps)
    lam = torch.empty(p, m, n, dtype=torch.float64, device='cuda')
    plan.heat_adjoint(None, None, steps, dev(c), lam)
    lhs = float(np.sum(c * host(Tv)))
    rhs = float(np.sum(host(lam) * v))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def _loss_fd(cyl, m, n, p, alpha, dt, steps, X0, g, tgt, wts):
    plan = cyl.Plan(m, n, p, alpha, dt, 1e-14, poisson=False, heat=True)
    T = dev(X0)
    plan.heat_step(T, dev(g), steps, g_step_stride=(p * m * n if g.ndim == 4 else 0))
    d = host(T) - tgt
    plan.close()
    return float(np.sum(wts * d * d))


def _halfcomplex_weights(p, m, n):
    """L = sum over the full complex coefficient array of |X - X_target|^2:
    weight 1 on slice 0 and the Nyquist slice, 2 on the Re/Im slices."""
    w = np.full((p, 1, 1), 2.0)
    w[0] = w[p - 1] = 1.0
    return np.broadcast_to(w, (p, m, n))


def test_gradients_match_central_differences(cyl):
    p, m, n, steps = 8, 17, 15, 12
    alpha, dt = 0.5, 1e-3
    rng = np.random.default_rng(44)
    X0 = inputs.smooth_coeffs(p, m, n, 1.25, rng)
    g = np.stack([inputs.smooth_coeffs(p, m, n, 1.25, rng) for _ in range(steps)])
    tgt = inputs.smooth_coeffs(p, m, n, 1.25, rng)
    wts = _halfcomplex_weights(p, m, n)
    plan = cyl.Plan(m, n, p, alpha, dt, 1e-14, poisson=False, heat=True)
    T = dev(X0)
    plan.heat_step(T, dev(g), steps, g_step_stride=p * m * n)
    lamN = 2.0 * wts * (host(T) - tgt)
    dT0 = torch.empty(p, m, n, dtype=torch.float64, device='cuda')
    dg = torch.empty(g.shape, dtype=torch.float64, device='cuda')
    dal = torch.zeros(1, dtype=torch.float64, device='cuda')
    plan.heat_adjoint(dev(X0), dev(g), steps, dev(lamN), dT0, dg, dal, g_step_stride=p * m * n, ckpt_every=4)
    dT0, dg, dal = host(dT0), host(dg), host(dal)[0]
    L = lambda a=alpha, x=X0, gg=g: _loss_fd(cyl, m, n, p, a, dt, steps, x, gg, tgt, wts)
    for which in ('X0', 'g'):
        d = rng.standard_normal(X0.shape if which == 'X0' else g.shape)
        h = 1e-3
        if which == 'X0':
            fd = (L(x=X0 + h * d) - L(x=X0 - h * d)) / (2 * h)
            an = float(np.sum(dT0 * d))
        else:
            fd = (L(gg=g + h * d) - L(gg=g - h * d)) / (2 * h)
            an = float(np.sum(dg * d))
        assert abs(fd - an) <= TOL_GRAD * abs(fd)
    h = 1e-4 * alpha
    fd = (L(a=alpha + h) - L(a=alpha - h)) / (2 * h)
    assert abs(fd - dal) <= TOL_GRAD * abs(fd)


def test_autograd_function(cyl):
    from paper_2206_04827_gb300.autograd import heat
    p, m, n, steps = 6, 12, 10, 5
    rng = np.random.default_rng(8)
    X0 = dev(inputs.smooth_coeffs(p, m, n, 1.3, rng)).requires_grad_(True)
    g = dev(inputs.smooth_coeffs(p, m, n, 1.3, rng)).requires_grad_(True)
    alpha = torch.tensor(0.4, dtype=torch.float64, device='cuda', requires_grad=True)
    T = heat(X0, g, alpha, 0.02, steps, ckpt_every=2)
    loss = (T * T).sum()
    loss.backward()
    Xh, gh = X0.detach().cpu().numpy(), g.detach().cpu().numpy()
    XN = oheat.heat_steps(Xh, gh, 0.4, 0.02, steps)
    w0, wg, wa = oheat.heat_adjoint(Xh, gh, 0.4, 0.02, steps, 2.0 * XN)
    assert rel(X0.grad.cpu().numpy(), w0) <= 1e-11
    assert rel(g.grad.cpu().numpy(), wg) <= 1e-11
    assert abs(alpha.grad.item() - wa) <= 1e-9 * abs(wa)


def test_adjoint_full_size_128_200_steps(cyl):
    """The 128^3 adjoint workload: alpha 0.5, dt 1e-3, 200 steps, checkpoint
    every 20, space-time forcing; gradients checked by central differences
    of the GPU forward along seeded directions (T0, g) and in alpha."""
    p = m = n = 128
    steps, every = 200, 20
    alpha, dt = 0.5, 1e-3
    rng = inputs.rng_for(1004)
    r = np.cos((m - 1 - np.arange(m)) * np.pi / (m - 1))
    th = (2 * np.arange(p) - p) * np.pi / p
    plan = cyl.Plan(m, n, p, alpha, dt, 1e-14, poisson=False, heat=True)
    T0 = plan.vals2coeffs(dev(inputs.eigenmode_values(r, r, th, inputs.eigenmode_list(8, rng))),
                          torch.empty(p, m, n, dtype=torch.float64, device='cuda'))
    g = torch.stack([dev(inputs.smooth_coeffs(p, m, n, 1.25, rng)) for _ in range(steps)])
    tgt = dev(inputs.smooth_coeffs(p, m, n, 1.25, rng))
    wts = dev(_halfcomplex_weights(p, m, n))
    N = p * m * n

    def loss(a=alpha, x=None, gg=None):
        pl = plan if a == alpha else cyl.Plan(m, n, p, a, dt, 1e-14, poisson=False, heat=True)
        T = (T0 if x is None else x).clone()
        pl.heat_step(T, g if gg is None else gg, steps, g_step_stride=N)
        d = T - tgt
        return float((wts * d * d).sum().item()), T

    L0, TN = loss()
    dT0 = torch.empty_like(T0)
    dg = torch.empty_like(g)
    dal = torch.zeros(1, dtype=torch.float64, device='cuda')
    plan.heat_adjoint(T0, g, steps, 2.0 * wts * (TN - tgt), dT0, dg, dal, g_step_stride=N, ckpt_every=every)
    plan.sync()
    d0 = dev(inputs.smooth_coeffs(p, m, n, 1.25, rng))
    h = 1e-3
    fd = (loss(x=T0 + h * d0)[0] - loss(x=T0 - h * d0)[0]) / (2 * h)
    assert abs(fd - float((dT0 * d0).sum())) <= TOL_GRAD * abs(fd)
    dgd = torch.stack([dev(inputs.smooth_coeffs(p, m, n, 1.25, rng)) for _ in range(steps)])
    fd = (loss(gg=g + h * dgd)[0] - loss(gg=g - h * dgd)[0]) / (2 * h)
    assert abs(fd - float((dg * dgd).sum())) <= TOL_GRAD * abs(fd)
    ha = 1e-4 * alpha
    fd = (loss(a=alpha + ha)[0] - loss(a=alpha - ha)[0]) / (2 * ha)
    assert abs(fd - dal.item()) <= TOL_GRAD * abs(fd)


@pytest.mark.parametrize('steps,every,wall', [(12, 4, False), (13, 5, False), (9, 3, True), (6, 6, False)])
def test_forward_checkpoints_give_identical_gradients(cyl, steps, every, wall):
    """The adjoint fed with the checkpoints its forward run wrote (cyl_heat_step's
    ckpt, same ckpt_every) skips its own checkpoint pass and returns the same
    gradients bit for bit (the states come from the same kernel arithmetic),
    with the smaller workspace."""
    p, m, n = 8, 17, 15
    alpha, dt = 0.45, 0.01
    X0, g, lamN = _problem(p, m, n, steps, 70 + steps, True)
    bc = dev(otr.coeffs2vals(inputs.smooth_coeffs(p, m, n, 1.2, np.random.default_rng(steps)))) if wall else None
    plan = cyl.Plan(m, n, p, alpha, dt, 1e-14, poisson=False, heat=True)
    N = p * m * n
    T = dev(X0)
    ck = torch.empty((steps // every + 1) * N, dtype=torch.float64, device='cuda')
    plan.heat_step(T, dev(g), steps, g_step_stride=N, ckpt=ck, ckpt_every=every, bc=bc)
    outs = []
    for ckpt in (None, ck):
        dT0 = torch.empty(p, m, n, dtype=torch.float64, device='cuda')
        dg = torch.empty(g.shape, dtype=torch.float64, device='cuda')
        dal = torch.zeros(1, dtype=torch.float64, device='cuda')
        nb = plan.adjoint_workspace_bytes(steps, every, True, have_ckpt=ckpt is not None)
        ws = torch.empty((nb + 7) // 8, dtype=torch.float64, device='cuda')
        plan.heat_adjoint(dev(X0), dev(g), steps, dev(lamN), dT0, dg, dal, g_step_stride=N, ckpt_every=every,
                          workspace=ws, bc=bc, ckpt=ckpt)
        plan.sync()
        outs.append((dT0, dg, dal))
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    assert plan.adjoint_workspace_bytes(steps, every, True, True) < plan.adjoint_workspace_bytes(steps, every, True)
