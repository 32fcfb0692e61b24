"""GPU Navier-Stokes step (cyl_ns_step, Section 4) against the oracle's
IMEX-BDF1 step in poloidal-toroidal form (oracle/ns.py) on the same seeded
vorticity states: the nonlinear forcing exercised by smooth states of
order-one amplitude, several steps, <= 1e-12 relative max-norm on the
coefficients; the 128^3 workload against extended-precision reference
values, with a bar derived from the FP64 rounding floor of the step; and the
plan checks (missing solvers, odd n_r)."""
import os

import numpy as np
import pytest

from oracle import ns as ons
from paper_2206_04827_gb300 import inputs

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

TOL_SOLVE = 1e-12
GOLD_NS = os.path.join(os.path.dirname(__file__), 'golden', 'ns128_sampled.npz')


@pytest.fixture(scope='module')
def cyl():
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    from paper_2206_04827_gb300 import cyl as C
    return C


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).cuda()


def relerr(got, want):
    return np.abs(got - want).max() / max(np.abs(want).max(), 1e-300)


@pytest.mark.parametrize('m,n,p,steps', [(12, 11, 8, 2), (16, 13, 12, 3), (24, 20, 16, 2)])
def test_ns_steps_match_oracle(cyl, m, n, p, steps):
    rng = np.random.default_rng(m * 10 + p)
    Lw = 3.0 * inputs.smooth_coeffs(p, m, n, 1.4, rng)
    Gw = 3.0 * inputs.smooth_coeffs(p, m, n, 1.4, rng)
    Re, dt = 20.0, 5e-3
    plan = cyl.Plan(m, n, p, 1.0 / Re, dt, 1e-14, poisson=True, heat=True, extra_flags=cyl.WITH_DISK)
    L, G = dev(Lw), dev(Gw)
    plan.ns_step(L, G, steps)
    plan.sync()
    want_l, want_g = ons.ns_steps(Lw, Gw, Re, dt, steps)
    # the step is not linear: the difference from the pure heat steps must be visible
    from oracle import heat as oheat
    lin = oheat.heat_steps(Lw, np.zeros_like(Lw), 1.0 / Re, dt, steps)
    assert relerr(want_l, lin) > 1e-6
    assert relerr(L.cpu().numpy(), want_l) <= TOL_SOLVE
    assert relerr(G.cpu().numpy(), want_g) <= TOL_SOLVE


def test_ns_128_bench_state_matches_oracle(cyl):
    """The Navier-Stokes workload at full size, in the bench's launch
    configuration (128^3, Re 100, dt 1e-3, ADI tolerance 1e-14, the bench's
    seeded potentials): one step against the oracle's extended-precision
    step on sampled slices and coefficients (tests/golden/make_ns128.py).
    The nonlinear term amplifies FP64 rounding: a plain FP64 evaluation of
    the same formulas (the oracle's FP64 step, error stored with the values)
    lands 3.8e-11 (lambda) and 2.4e-13 (gamma) of the field's maximum from
    the reference, so the bar is 4x that floor, and never looser than 1e-12
    where the floor is below it."""
    ref = np.load(GOLD_NS)
    L = 128
    rng = inputs.rng_for(int(ref['seed']))
    Lw = inputs.smooth_coeffs(L, L, L, float(ref['decay']), rng)
    Gw = inputs.smooth_coeffs(L, L, L, float(ref['decay']), rng)
    Re, dt = float(ref['Re']), float(ref['dt'])
    plan = cyl.Plan(L, L, L, 1.0 / Re, dt, 1e-14, poisson=True, heat=True, extra_flags=cyl.WITH_DISK)
    l, g = dev(Lw), dev(Gw)
    plan.ns_step(l, g, 1)
    plan.sync()
    sl = torch.as_tensor(ref['slices'], device='cuda')
    idx = torch.as_tensor(ref['idx'], device='cuda')
    pick = lambda X: X.index_select(0, sl).index_select(1, idx).index_select(2, idx).cpu().numpy()
    el = np.abs(pick(l) - ref['lam']).max() / float(ref['lam_max'])
    eg = np.abs(pick(g) - ref['gam']).max() / float(ref['gam_max'])
    tl = max(TOL_SOLVE, 4.0 * float(ref['fp64_err_lam']))
    tg = max(TOL_SOLVE, 4.0 * float(ref['fp64_err_gam']))
    print('ns128 one step vs extended-precision reference: lambda %.2e (bar %.1e), gamma %.2e (bar %.1e)'
          % (el, tl, eg, tg))
    assert el <= tl and eg <= tg


def test_ns_step_needs_every_solver_and_even_radial_grid(cyl):
    x = torch.zeros(8 * 12 * 9, dtype=torch.float64, device='cuda')
    noheat = cyl.Plan(12, 9, 8, 0.1, 1e-2, 1e-12, poisson=True, heat=False, extra_flags=cyl.WITH_DISK)
    with pytest.raises(cyl.CylError) as ei:
        noheat.ns_step(x, x, 1)
    assert ei.value.status == cyl.ESTATE
    odd = cyl.Plan(11, 9, 8, 0.1, 1e-2, 1e-12, poisson=True, heat=True, extra_flags=cyl.WITH_DISK)
    with pytest.raises(cyl.CylError) as ei:
        odd.ns_step(x, x, 1)
    assert ei.value.status == cyl.EINVAL
