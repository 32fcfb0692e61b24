"""Host-side logic of libcyl, run on the CPU through the C ABI (no device
calls): exported symbols, elliptic functions, the plan's operator blocks
against the oracle, spectral intervals, Zolotarev shifts and their ADI
convergence, and argument validation."""
import os
import re

import numpy as np
import pytest
from scipy import special

from oracle import sylvester as sy

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope='module')
def cyl():
    from paper_2206_04827_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    from paper_2206_04827_gb300 import cyl as C
    return C


def _header_functions():
    txt = open(os.path.join(ROOT, 'include', 'cyl.h')).read()
    txt = re.sub(r'/\*.*?\*/', '', txt, flags=re.S)
    return sorted(set(re.findall(r'\b(cyl_[A-Za-z0-9_]+)\s*\(', txt)))


def test_library_exports_every_declared_function(cyl):
    names = _header_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(cyl._lib, name), name
    assert set(cyl.exported_symbols()) <= set(names)


@pytest.mark.parametrize('kp', [0.9, 0.5, 1e-2, 1e-4, 1e-6, 1e-9])
def test_elliptic_functions_match_high_precision(cyl, kp):
    """K against scipy, K and dn against 40-digit mpmath (scipy's dn loses
    digits near u = K when k' is small)."""
    mp = pytest.importorskip('mpmath')
    mp.mp.dps = 40
    K = cyl.ellip_K(kp)
    assert K == pytest.approx(special.ellipkm1(kp * kp), rel=1e-13)
    m = 1 - mp.mpf(kp) ** 2
    assert K == pytest.approx(float(mp.ellipk(m)), rel=1e-14)
    for frac in (0.0, 0.1, 0.37, 0.5, 0.8, 0.97):
        u = frac * K
        assert cyl.jacobi_dn(u, kp) == pytest.approx(float(mp.ellipfun('dn', u, m=m)), rel=1e-12)


@pytest.mark.parametrize('kp', [1e-5, 1e-8, 4e-9, 1e-12])
def test_dn_identities_for_tiny_complementary_modulus(cyl, kp):
    """dn(0) = 1, dn(K) = k', dn(u) dn(K - u) = k' (DLMF 22.5, 22.4)."""
    K = cyl.ellip_K(kp)
    assert K == pytest.approx(np.log(4.0 / kp), rel=1e-6)
    assert cyl.jacobi_dn(0.0, kp) == pytest.approx(1.0, rel=1e-15)
    assert cyl.jacobi_dn(K, kp) == pytest.approx(kp, rel=1e-10)
    for frac in (0.05, 0.3, 0.5, 0.71, 0.99):
        u = frac * K
        assert cyl.jacobi_dn(u, kp) * cyl.jacobi_dn(K - u, kp) == pytest.approx(kp, rel=1e-10)


def _blocks(ms, pr, pz):
    ir = np.arange(pr, ms.m - 2, 2)
    iz = np.arange(pz, ms.n - 2, 2)
    return (ms.A[np.ix_(ir, ir)], ms.C[np.ix_(ir, ir)], ms.B[np.ix_(iz, iz)], ms.D[np.ix_(iz, iz)])


@pytest.mark.parametrize('m,n,p', [(9, 8, 6), (12, 13, 8), (33, 20, 4)])
def test_plan_operators_equal_oracle_blocks(cyl, m, n, p):
    alpha, dt = 0.7, 0.01
    plan = cyl.Plan(m, n, p, alpha, dt, 1e-13, poisson=True, heat=True, both_parities=True, host_only=True)
    for which, kind, ka in ((0, 'poisson', None), (1, 'heat', alpha * dt)):
        for k in range(p // 2 + 1):
            ms = sy.ModeSystem(m, n, k, kind, ka)
            for par in (0, 1):
                A, C, B, D = _blocks(ms, par, par)
                assert np.allclose(plan.operator(0, which, k, par), A, atol=1e-12 * np.abs(A).max())
                assert np.allclose(plan.operator(1, which, k, par), C, atol=1e-14)
                assert np.allclose(plan.operator(2, which, k, par), B, atol=1e-14)
                assert np.allclose(plan.operator(3, which, k, par), D, atol=1e-12 * max(np.abs(D).max(), 1))
    plan.close()


@pytest.mark.parametrize('m,n,p', [(17, 17, 8), (33, 33, 32), (64, 48, 16)])
def test_intervals_contain_spectra_and_shifts_lie_inside(cyl, m, n, p):
    alpha, dt = 1.0, 1e-3
    plan = cyl.Plan(m, n, p, alpha, dt, 1e-14, poisson=True, heat=True, host_only=True)
    for which, kind, ka in ((0, 'poisson', None), (1, 'heat', alpha * dt)):
        for k in sorted({0, 1, 2, p // 4, p // 2}):
            par = k % 2
            J, (a, b, c, d), ps, qs = plan.shifts(which, k, par)
            ms = sy.ModeSystem(m, n, k, kind, ka)
            for pz in (0, 1):
                A, C, B, D = _blocks(ms, par, pz)
                eP = np.linalg.eigvals(np.linalg.solve(C, A))
                eQ = -np.linalg.eigvals(np.linalg.solve(B, D))
                assert np.abs(eP.imag).max() < 1e-6 * np.abs(eP).max()
                assert a <= eP.real.min() and eP.real.max() <= b
                assert c <= eQ.real.min() and eQ.real.max() <= d
            assert np.all((qs >= a) & (qs <= b)) and np.all((ps >= c) & (ps <= d))
            gam = abs(c - a) * abs(d - b) / (abs(c - b) * abs(d - a))
            assert J == int(np.ceil(np.log(16 * gam) * np.log(4 / 1e-14) / np.pi ** 2))
    plan.close()


def _adi(A, B, C, D, E, ps, qs):
    """Algorithm 1 with the plan's shifts (host-side convention check)."""
    U = np.zeros_like(E)
    for j in range(len(ps)):
        p_, q_ = ps[j], qs[j]
        Z = np.linalg.solve(A - p_ * C, (q_ - p_) * E + (A - q_ * C) @ U)
        X = np.linalg.solve(D + q_ * B, Z.T).T
        U = X @ (D + (ps[j + 1] if j + 1 < len(ps) else 0.0) * B).T
    return X


@pytest.mark.parametrize('kind', ['poisson', 'heat'])
def test_plan_shifts_make_adi_converge_to_direct_solve(cyl, kind):
    m, n, p = 40, 36, 8
    alpha, dt = 0.5, 2e-3
    plan = cyl.Plan(m, n, p, alpha, dt, 1e-13, poisson=True, heat=True, host_only=True)
    which = 0 if kind == 'poisson' else 1
    rng = np.random.default_rng(4)
    for k in (0, 3, 4):
        par = k % 2
        J, _, ps, qs = plan.shifts(which, k, par)
        for pz in (0, 1):
            A, C, B, D = (plan.operator(o, which, k, pz if o > 1 else par) for o in range(4))
            ii, jj = np.meshgrid(np.arange(A.shape[0]), np.arange(B.shape[0]), indexing='ij')
            E = rng.standard_normal(ii.shape) * 1.3 ** (-(ii + jj))
            X = _adi(A, B, C, D, E, ps, qs)
            Xd = sy.solve_kron(A, B, C, D, E)
            assert np.abs(X - Xd).max() < 1e-12 * np.abs(Xd).max()
    plan.close()


def test_argument_validation(cyl):
    bad = [dict(n_r=3, n_z=8, n_theta=8), dict(n_r=8, n_z=3, n_theta=8), dict(n_r=8, n_z=8, n_theta=7),
           dict(n_r=8, n_z=8, n_theta=0), dict(n_r=8, n_z=8, n_theta=8, adi_tol=0.5),
           dict(n_r=8, n_z=8, n_theta=8, adi_tol=0.0), dict(n_r=8, n_z=8, n_theta=8, heat=True, alpha=-1.0, dt=0.1),
           dict(n_r=8, n_z=8, n_theta=8, heat=True, alpha=1.0, dt=0.0), dict(n_r=8, n_z=8, n_theta=8, poisson=False)]
    for kw in bad:
        kw.setdefault('adi_tol', 1e-12)
        with pytest.raises(cyl.CylError) as ei:
            cyl.Plan(host_only=True, **kw)
        assert ei.value.status == cyl.EINVAL
    plan = cyl.Plan(8, 8, 8, host_only=True)
    with pytest.raises(cyl.CylError) as ei:
        plan.shifts(1, 0, 0)
    assert ei.value.status == cyl.ESTATE
    assert cyl.status_string(cyl.ETIMEOUT).startswith('CYL_ETIMEOUT')


def test_bdf_plan_builds_every_order_with_its_kappa(cyl):
    """A BDF 4 plan holds the step operators of orders 1..4, each the oracle's
    eq. HelmholtzMatEqn block with kappa = kappa^(b) h (Section 3 BDF
    definitions), and shifts that make Algorithm 1 converge for each."""
    from oracle import heat as oheat
    m, n, p = 20, 18, 8
    alpha, dt = 0.9, 4e-3
    plan = cyl.Plan(m, n, p, alpha, dt, 1e-13, poisson=False, heat=True, host_only=True, bdf_order=4)
    rng = np.random.default_rng(6)
    for b in (1, 2, 3, 4):
        ka = alpha * dt * float(oheat.bdf_coefficients(b)[0])
        for k in (0, 3):
            par = k % 2
            ms = sy.ModeSystem(m, n, k, 'heat', ka)
            A, C, B, D = _blocks(ms, par, 0)
            assert np.allclose(plan.operator(0, b, k, par), A, atol=1e-12 * np.abs(A).max())
            assert np.allclose(plan.operator(3, b, k, 0), D, atol=1e-12 * max(np.abs(D).max(), 1))
            J, _, ps, qs = plan.shifts(b, k, par)
            E = rng.standard_normal((A.shape[0], B.shape[0]))
            X = _adi(A, B, C, D, E, ps, qs)
            Xd = sy.solve_kron(A, B, C, D, E)
            assert np.abs(X - Xd).max() < 1e-11 * np.abs(Xd).max()
    with pytest.raises(cyl.CylError):
        plan.shifts(5, 0, 0)
    plan.close()
    # a BDF1 plan has no higher-order tables; orders outside 1..4 are rejected
    p1 = cyl.Plan(m, n, p, alpha, dt, 1e-13, poisson=False, heat=True, host_only=True)
    with pytest.raises(cyl.CylError) as ei:
        p1.shifts(2, 0, 0)
    assert ei.value.status == cyl.ESTATE
    for bad in (0, 5):
        with pytest.raises(cyl.CylError) as ei:
            cyl.Plan(m, n, p, alpha, dt, 1e-13, poisson=False, heat=True, host_only=True, bdf_order=bad)
        assert ei.value.status == cyl.EINVAL


def _radial_column(rec, R, U, f, first, k):
    """One column of the radial sweep from the plan's records (the kernel's
    arithmetic order is not reproduced, only its algebra)."""
    M = len(f)
    y = f.copy()
    if not first:
        for i in range(M):
            for o in range(-2, 4):
                if 0 <= i + o < M:
                    y[i] += rec[i, o + 2] * U[i + o]
    z = np.zeros(M + 3)
    w = np.zeros(M)
    top = M if k == 0 else k
    for i in range(top):
        w[i] = y[i] + (rec[i, 6] * w[i - 1] if i >= 1 else 0) + (rec[i, 7] * w[i - 2] if i >= 2 else 0)
    if k:
        v = np.zeros(M + 3)
        for i in range(M - 1, k + 2, -1):
            v[i] = y[i] + rec[i, 6] * v[i + 1] + rec[i, 7] * v[i + 2] + rec[i, 8] * v[i + 3]
        rhs = np.array([w[k - 2], w[k - 1], y[k], y[k + 1], y[k + 2], v[k + 3], v[k + 4], v[k + 5]])
        z[k:k + 3] = R.reshape(3, 8) @ rhs
        for i in range(k + 3, M):
            z[i] = rec[i, 11] * v[i] + rec[i, 9] * z[i - 1] + rec[i, 10] * z[i - 2]
    for i in range(top - 1, -1, -1):
        z[i] = rec[i, 11] * w[i] + rec[i, 8] * z[i + 1] + rec[i, 9] * z[i + 2] + rec[i, 10] * z[i + 3]
    return z[:M]


def _vertical_row(rec, R, zrow, k):
    Nz = len(zrow)
    x = np.zeros(Nz + 2)
    w = np.zeros(Nz)
    top = Nz if k == 0 else k
    for c in range(top):
        w[c] = zrow[c] + (rec[c, 0] * w[c - 1] if c >= 1 else 0)
    if k:
        v = np.zeros(Nz + 2)
        for c in range(Nz - 1, k + 1, -1):
            v[c] = zrow[c] + rec[c, 0] * v[c + 1] + rec[c, 1] * v[c + 2]
        xi = R[:15].reshape(3, 5) @ np.array([w[k - 1], zrow[k], zrow[k + 1], v[k + 2], v[k + 3]])
        x[k:k + 2] = xi[:2]
        for c in range(k + 2, Nz):
            x[c] = rec[c, 3] * v[c] + rec[c, 2] * x[c - 1]
        assert abs(x[k + 2] - xi[2]) <= 1e-10 * max(1.0, np.abs(xi).max())
    for c in range(top - 1, -1, -1):
        x[c] = rec[c, 3] * w[c] + rec[c, 1] * x[c + 1] + rec[c, 2] * x[c + 2]
    x = x[:Nz]
    u = np.zeros(Nz)
    for c in range(Nz):
        for o in range(-1, 3):
            if 0 <= c + o < Nz:
                u[c] += rec[c, 5 + o] * x[c + o]
    return x, u


@pytest.mark.parametrize('which', [0, 1, 4])
def test_item_tables_drive_adi_to_the_direct_solve(cyl, which):
    """Algorithm 1 run from the plan's own factor records (plain LU sweeps and
    the twisted two-sided sweeps with their interface maps) reaches the direct
    solution of every item's block Sylvester equation."""
    m, n, p = 40, 36, 8
    plan = cyl.Plan(m, n, p, 0.6, 2e-3, 1e-13, poisson=True, heat=True, host_only=True, bdf_order=4)
    rng = np.random.default_rng(3 + which)
    seen_twisted = False
    nitems = 0
    while True:
        try:
            info, _, _ = plan.item_tables(which, nitems, 0)
        except cyl.CylError:
            break
        nitems += 1
    assert nitems > 0
    for item in range(0, nitems, 3):
        kr, kz = _drive_item_to_direct_solve(cyl, plan, which, item, rng)
        seen_twisted |= bool(kr and kz)
    assert seen_twisted
    plan.close()


def _drive_item_to_direct_solve(cyl, plan, which, item, rng):
    """Algorithm 1 on one item from its factor records against the dense
    Kronecker solve of its block equation; returns the twisted splits."""
    info, _, _ = plan.item_tables(which, item, 0)
    M, Nz, J, kr, kz = info['M'], info['Nz'], info['J'], info['twr'], info['twz']
    A, C = plan.operator(0, which, info['k'], info['pr']), plan.operator(1, which, info['k'], info['pr'])
    B, D = plan.operator(2, which, info['k'], info['pz']), plan.operator(3, which, info['k'], info['pz'])
    ii, jj = np.meshgrid(np.arange(M), np.arange(Nz), indexing='ij')
    E = rng.standard_normal((M, Nz)) * 1.3 ** (-(ii + jj))
    U = np.zeros((M, Nz))
    X = None
    for j in range(J):
        _, rad, ver = plan.item_tables(which, item, j)
        rrec, Rr = rad[:M * 12].reshape(M, 12), rad[M * 12:]
        vrec, Rz = ver[:Nz * 8].reshape(Nz, 8), ver[Nz * 8:]
        Z = np.stack([_radial_column(rrec, Rr, U[:, c], E[:, c], j == 0, kr) for c in range(Nz)], axis=1)
        rows = [_vertical_row(vrec, Rz, Z[a], kz) for a in range(M)]
        X = np.stack([r[0] for r in rows])
        U = np.stack([r[1] for r in rows])
    Xd = sy.solve_kron(A, B, C, D, E)
    assert np.abs(X - Xd).max() < 1e-11 * np.abs(Xd).max(), (item, kr, kz)
    return kr, kz


def test_cluster_plans_twist_every_item(cyl):
    """Cluster plans (several CTAs per item, at most 128 chains each) carry
    twisted two-sided solves on items whose chains exceed what one CTA
    twists, and Algorithm 1 from those records still reaches the direct
    solve; without cluster mode such items keep one-sided LU records."""
    m, n, p = 140, 132, 8
    plain = cyl.Plan(m, n, p, 0.6, 2e-3, 1e-13, poisson=True, heat=True, host_only=True)
    info, _, _ = plain.item_tables(1, 0, 0)
    assert info['twr'] == 0 and info['twz'] == 0
    plain.close()
    plan = cyl.Plan(m, n, p, 0.6, 2e-3, 1e-13, poisson=True, heat=True, host_only=True,
                    extra_flags=cyl.FORCE_CLUSTER)
    li = plan.launch_info(1)
    assert li['ctas_per_item'] > 1 and li['all_twisted'] == 0          # cluster launches keep their own kernel
    rng = np.random.default_rng(17)
    for which, item in ((0, 0), (1, 3)):
        kr, kz = _drive_item_to_direct_solve(cyl, plan, which, item, rng)
        assert kr > 0 and kz > 0
    plan.close()


@pytest.mark.parametrize('mnp,flags,want', [
    ((512, 512, 512), 0, (1, 256, 512, 0)),          # two-slice arrays leave shared memory: twisted single slices
    ((512, 512, 512), 'plain', (2, 0, 512, 0)),
    ((300, 300, 4), 0, (1, 160, 320, 0)),
    ((256, 256, 256), 0, (1, 128, 256, 1)),          # a single slice's iterate fits shared memory
    ((128, 128, 128), 0, (2, 128, 256, 2)),          # two-slice items in shared memory, twisted
    ((128, 128, 128), 'plain', (2, 0, 128, 2)),
    ((20, 19, 8), 'global', (1, 32, 64, 0)),         # radial class 9: one-sided radial, not all twisted
    ((8, 520, 4), 0, (2, 0, 512, 1)),                # 518 radial chains on 512 threads
    ((600, 600, 8), 0, (2, 0, 512, 0)),              # class sizes above 256: one-sided, threads loop
])
def test_launch_layouts(cyl, mnp, flags, want):
    """(slices per item, twisted half, threads, placement) of the heat
    kernel's launch as the plan chooses it."""
    extra = {0: 0, 'plain': cyl.PLAIN_SWEEPS, 'global': cyl.FORCE_GLOBAL}[flags]
    plan = cyl.Plan(*mnp, 0.1, 1e-4, 1e-14, poisson=True, heat=True, host_only=True, extra_flags=extra)
    li = plan.launch_info(1)
    assert (li['slices'], li['twist_half'], li['threads'], li['placement']) == want, li
    assert li['built'] == 1 and li['ctas_per_item'] == 1 and li['smem'] <= 226 * 1024
    # single-slice twisted layouts of large grids: every item twisted both ways
    assert li['all_twisted'] == (1 if (want[0] == 1 and want[1] >= 128) else li['all_twisted'])
    m, n, p = mnp
    h = p // 2
    pairs = h - 1
    assert li['items'] == 2 * ((2 * pairs if want[0] == 1 else pairs) + 2)   # x 2 vertical parity classes
    plan.close()


def test_batch_configuration_on_host(cyl):
    """Host-only batch plan of uneven grids: a feasible default (threshold,
    groups) is chosen at plan time, every accepted setting assigns all
    items to the two classes, twisted groups split pairs into single slices
    (more items than with one-sided sweeps), and device calls are refused."""
    rng = np.random.default_rng(12)
    k = 40
    n_r, n_z = rng.integers(16, 200, size=k), rng.integers(16, 200, size=k)
    n_t, alpha = rng.choice([8, 16, 32], size=k), rng.uniform(0.05, 1.0, size=k)
    tw = cyl.BatchPlan(n_r, n_z, n_t, alpha, 1e-3, 1e-13, host_only=True)
    pl = cyl.BatchPlan(n_r, n_z, n_t, alpha, 1e-3, 1e-13, host_only=True, plain_sweeps=True)
    thr, G, counts = tw.config()
    assert G in (1, 2, 4) and sum(counts) > 0
    accepted = 0
    for th in (0, 31, 63, 95):
        for G in (1, 2, 4):
            for bp in (tw, pl):
                try:
                    bp.set_config(th, G)
                except cyl.CylError as e:
                    assert e.status == cyl.EINVAL
                    continue
                accepted += 1
                t2, g2, c2 = bp.config()
                assert (t2, g2) == (th, G) and min(c2) >= 0 and sum(c2) > 0
    assert accepted >= 8
    tw.set_config(0, 1)
    pl.set_config(0, 1)
    assert tw.config()[2][0] > pl.config()[2][0]
    # two chains per thread in the one-sided classes; other values are refused
    pl.set_config(31, 2, chains_per_thread=2)
    assert pl.chains_per_thread() == 2 and pl.config()[:2] == (31, 2)
    for bad in (0, 3):
        with pytest.raises(cyl.CylError):
            pl.set_config(31, 2, chains_per_thread=bad)
    import torch
    x = torch.zeros(1, dtype=torch.float64)
    with pytest.raises((cyl.CylError, ValueError)):
        tw.heat_step(x, None, 1)


@pytest.mark.parametrize('which,flags', [(1, 0), (3, 0), (1, 'cluster')])
def test_transposed_item_tables_drive_adi_to_the_direct_solve(cyl, which, flags):
    """The adjoint's records -- the forward-layout records of the flipped
    transposes J A^T J, J C^T J, J B^T J, J D^T J, twisted where the forward
    records are (one-sided in cluster plans) -- drive Algorithm 1, run on the
    index-reversed right side, to the direct solution of the transposed
    system A^T X B + C^T X D = E with the same shifts, for the BDF1 and the
    BDF3 step."""
    m, n, p = 30, 26, 8
    extra = cyl.FORCE_CLUSTER if flags == 'cluster' else 0
    plan = cyl.Plan(m, n, p, 0.6, 2e-3, 1e-13, poisson=False, heat=True, host_only=True, bdf_order=3,
                    extra_flags=extra)
    rng = np.random.default_rng(21 + which)
    item = 0
    checked = twisted = 0
    while True:
        try:
            info, _, _ = plan.item_tables(which, item, 0, transposed=True)
        except cyl.CylError:
            break
        if item % 3 == 0:
            M, Nz, J, kr, kz = info['M'], info['Nz'], info['J'], info['twr'], info['twz']
            twisted += bool(kr and kz)
            A, C = plan.operator(0, which, info['k'], info['pr']), plan.operator(1, which, info['k'], info['pr'])
            B, D = plan.operator(2, which, info['k'], info['pz']), plan.operator(3, which, info['k'], info['pz'])
            ii, jj = np.meshgrid(np.arange(M), np.arange(Nz), indexing='ij')
            E = rng.standard_normal((M, Nz)) * 1.3 ** (-(ii + jj))
            Er = E[::-1, ::-1].copy()
            U = np.zeros((M, Nz))
            for j in range(J):
                _, rad, ver = plan.item_tables(which, item, j, transposed=True)
                rrec, Rr = rad[:M * 12].reshape(M, 12), rad[M * 12:]
                vrec, Rz = ver[:Nz * 8].reshape(Nz, 8), ver[Nz * 8:]
                Z = np.stack([_radial_column(rrec, Rr, U[:, c], Er[:, c], j == 0, kr) for c in range(Nz)], axis=1)
                rows = [_vertical_row(vrec, Rz, Z[a], kz) for a in range(M)]
                X = np.stack([r[0] for r in rows])
                U = np.stack([r[1] for r in rows])
            Xd = sy.solve_kron(A.T, B.T, C.T, D.T, E)
            assert np.abs(X[::-1, ::-1] - Xd).max() < 1e-11 * np.abs(Xd).max(), item
            checked += 1
        item += 1
    assert checked >= 3
    assert (twisted == 0) if flags == 'cluster' else (twisted == checked)
    with pytest.raises(cyl.CylError) as ei:
        cyl.Plan(m, n, p, host_only=True).item_tables(0, 0, 0, transposed=True)
    assert ei.value.status == cyl.ESTATE


@pytest.mark.parametrize('k', [0, 1, 2, 5])
def test_pencil_spectra_are_the_dirichlet_eigenvalues(cyl, k):
    """The radial pencil of the Poisson step (A = -L_k against the R_2 block
    C) has as its smallest eigenvalue the first Dirichlet eigenvalue of the
    disk mode, j_{k,1}^2 (Bessel zero), and the vertical pencil (D = -D2
    against the C02 block B) pi^2 / 4; the plan's padded intervals enclose
    both (the spectra behind the shift choice of Algorithm 1)."""
    m, n, p = 64, 48, 16
    ms = sy.ModeSystem(m, n, k, 'poisson')
    A, C, B, D = _blocks(ms, k % 2, 0)
    mu = np.sort(np.linalg.eigvals(np.linalg.solve(C, A)).real)
    nu = np.sort(np.linalg.eigvals(np.linalg.solve(B, D)).real)     # D = -D2 for Poisson
    j1 = special.jn_zeros(k, 1)[0]
    assert abs(mu[0] - j1 ** 2) < 1e-9 * j1 ** 2
    assert abs(nu[0] - np.pi ** 2 / 4) < 1e-9
    plan = cyl.Plan(m, n, p, poisson=True, host_only=True)
    _, (a, b, c, d), _, _ = plan.shifts(0, k, k % 2)
    assert a <= j1 ** 2 <= b and a >= 0.9 * j1 ** 2
    assert c <= -np.pi ** 2 / 4 <= d and d <= -0.9 * np.pi ** 2 / 4
