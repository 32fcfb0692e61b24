"""GPU parity of the horizontal (disk) Poisson solve (Section 4, eq.
ptpoisson) through the C ABI against the oracle, plus a Bessel
eigenfunction of -Delta_h recovered on the GPU."""
import numpy as np
import pytest
from scipy import special

from oracle import disk as odisk, grid, transforms as otr
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


@pytest.mark.parametrize('m,n,p', [(5, 6, 4), (9, 8, 6), (16, 17, 8), (33, 33, 32), (40, 37, 16)])
def test_disk_poisson_coeffs_match_oracle(cyl, m, n, p):
    F = inputs.smooth_coeffs(p, m, n, 1.2, np.random.default_rng(m * 7 + n))
    plan = cyl.Plan(m, n, p, poisson=False, extra_flags=cyl.WITH_DISK)
    u = plan.disk_poisson(dev(F), torch.empty(p, m, n, dtype=torch.float64, device='cuda'), cyl.COEFFS)
    assert relerr(host(u), odisk.horizontal_poisson(F)) <= TOL_SOLVE


def test_disk_poisson_values_in_place(cyl):
    p, m, n = 16, 24, 19
    f = otr.coeffs2vals(inputs.smooth_coeffs(p, m, n, 1.2, np.random.default_rng(3)))
    plan = cyl.Plan(m, n, p, poisson=True, extra_flags=cyl.WITH_DISK)
    fu = dev(f)
    got = host(plan.disk_poisson(fu, fu, cyl.VALUES))
    want = otr.coeffs2vals(odisk.horizontal_poisson(otr.vals2coeffs(f)))
    assert relerr(got, want) <= TOL_SOLVE


def test_disk_poisson_both_parities_rough_data(cyl):
    p, m, n = 8, 14, 11
    F = np.random.default_rng(5).standard_normal((p, m, n))
    plan = cyl.Plan(m, n, p, poisson=False, both_parities=True, extra_flags=cyl.WITH_DISK)
    u = plan.disk_poisson(dev(F), torch.empty(p, m, n, dtype=torch.float64, device='cuda'), cyl.COEFFS)
    assert relerr(host(u), odisk.horizontal_poisson(F)) <= 1e-11


def test_disk_poisson_128_cubed_sampled_slices(cyl):
    p = m = n = 128
    F = inputs.smooth_coeffs(p, m, n, 1.25, np.random.default_rng(128))
    plan = cyl.Plan(m, n, p, poisson=False, extra_flags=cyl.WITH_DISK)
    u = host(plan.disk_poisson(dev(F), torch.empty(p, m, n, dtype=torch.float64, device='cuda'), cyl.COEFFS))
    slices = [0, 1, 2, 63, 64, 126, 127]
    want = odisk.horizontal_poisson(F, slices=slices)
    assert relerr(u[slices], want[slices]) <= TOL_SOLVE


def test_bessel_eigenfunction_on_gpu(cyl):
    p, m, n = 16, 33, 9
    mu, nu = 2, 1
    j = special.jn_zeros(mu, nu)[-1]
    TH, RR, ZZ = np.meshgrid(grid.theta_points(p), grid.cheb_points(m), grid.cheb_points(n), indexing='ij')
    u = special.jv(mu, j * RR) * np.cos(mu * TH) * np.exp(ZZ)
    plan = cyl.Plan(m, n, p, poisson=False, extra_flags=cyl.WITH_DISK)
    got = host(plan.disk_poisson(dev(j ** 2 * u), torch.empty(p, m, n, dtype=torch.float64, device='cuda'),
                                 cyl.VALUES))
    assert np.abs(got - u).max() < 1e-11 * np.abs(u).max()


def test_disk_needs_its_flag(cyl):
    plan = cyl.Plan(9, 8, 4)
    x = torch.zeros(4, 9, 8, dtype=torch.float64, device='cuda')
    with pytest.raises(cyl.CylError) as ei:
        plan.disk_poisson(x, x)
    assert ei.value.status == cyl.ESTATE
