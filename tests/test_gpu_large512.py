"""The 512^3 workload at full size, in the launch configuration the bench
times (one Poisson solve of f, then 20 BDF1 heat steps with alpha 0.1,
dt 1e-4 and forcing f from its solution; ADI tolerance 1e-15, where 1e-14
ends at 1.7e-12 after the 20 steps), compared on
sampled slices and coefficients with oracle values written by
tests/golden/make_large512.py (refined QZ solves; the file stores the
sampling)."""
import os

import numpy as np
import pytest

from paper_2206_04827_gb300 import inputs

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

TOL_SOLVE = 1e-12
GOLD = os.path.join(os.path.dirname(__file__), 'golden', 'large512_sampled.npz')


@pytest.fixture(scope='module')
def cyl():
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    from paper_2206_04827_gb300 import cyl as C
    return C


def test_large512_poisson_then_heat_matches_oracle(cyl):
    ref = np.load(GOLD)
    p = m = n = 512
    f = torch.as_tensor(inputs.smooth_coeffs(p, m, n, 1.1, inputs.rng_for(int(ref['seed']))), device='cuda')
    plan = cyl.Plan(m, n, p, float(ref['alpha']), float(ref['dt']), 1e-15, poisson=True, heat=True)
    T = torch.empty_like(f)
    plan.poisson(f, T, cyl.COEFFS)
    sl = torch.as_tensor(ref['slices'], device='cuda')
    idx = torch.as_tensor(ref['idx'], device='cuda')
    u = T.index_select(0, sl).index_select(1, idx).index_select(2, idx).cpu().numpy()
    plan.heat_step(T, f, int(ref['hsteps']))
    h = T.index_select(0, sl).index_select(1, idx).index_select(2, idx).cpu().numpy()
    plan.sync()
    errs = [np.abs(got - want).max() / np.abs(want).max() for got, want in ((u, ref['poisson']), (h, ref['heat']))]
    assert max(errs) <= TOL_SOLVE, errs
