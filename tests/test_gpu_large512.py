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


@pytest.mark.parametrize('layout', ['default', 'plain'])
def test_large512_poisson_then_heat_matches_oracle(cyl, layout):
    """default: single-slice items with twisted solves (2 x 256 threads, the
    bench's launch); plain: two-slice items with one-sided sweeps."""
    ref = np.load(GOLD)
    p = m = n = 512
    f = torch.as_tensor(inputs.smooth_coeffs(p, m, n, 1.1, inputs.rng_for(int(ref['seed']))), device='cuda')
    plan = cyl.Plan(m, n, p, float(ref['alpha']), float(ref['dt']), 1e-15, poisson=True, heat=True,
                    extra_flags=cyl.PLAIN_SWEEPS if layout == 'plain' else 0)
    li = plan.launch_info(1)
    want = (1, 256, 512) if layout == 'default' else (2, 0, 512)
    assert (li['slices'], li['twist_half'], li['threads']) == want, li
    T = torch.empty_like(f)
    plan.poisson(f, T, cyl.COEFFS)
    sl = torch.as_tensor(ref['slices'], device='cuda')
    idx = torch.as_tensor(ref['idx'], device='cuda')
    u = T.index_select(0, sl).index_select(1, idx).index_select(2, idx).cpu().numpy()
    plan.heat_step(T, f, int(ref['hsteps']))
    h = T.index_select(0, sl).index_select(1, idx).index_select(2, idx).cpu().numpy()
    plan.sync()
    errs = [np.abs(got - want).max() / np.abs(want).max() for got, want in ((u, ref['poisson']), (h, ref['heat']))]
    print('512^3 %s layout vs oracle: poisson %.2e, after the heat steps %.2e' % (layout, errs[0], errs[1]))
    assert max(errs) <= TOL_SOLVE, errs
