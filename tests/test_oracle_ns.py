"""Pins of the oracle's Navier-Stokes step in poloidal-toroidal form
(Section 4, eqs. ns, pt, ptpoisson, ptcurl, NSrewrite), each against an
independent computation in CARTESIAN components by sympy (curls and cross
products of Cartesian vector fields, projected on r-hat and theta-hat at the
grid points), so that a sign, a factor 1/r or a transposed derivative in the
cylindrical formulas of the oracle fails:

* spectral derivatives d_r, d_z, d_theta on a polynomial field;
* eq. pt: the components of curl(lambda z) + curl curl(gamma z);
* eq. ptpoisson's right sides z . curl N and z . curl curl N for a given N;
* the whole nonlinear term of a manufactured vortical flow (potentials
  chosen so that every field is a polynomial the grid resolves exactly);
* the recovery of (lambda, gamma) from a PT field by the two horizontal
  solves (eq. ptpoisson);
* quadratic scaling of the nonlinear term, and the linear limit of a step
  (small amplitude: the step is the heat step of Section 3, eq. NSrewrite);
* the extended-precision path that writes reference values: its transforms
  (round trip to 1e-17) and derivative matrix against the FP64 ones and
  against exact values, the manufactured flow, agreement with the FP64 step.
"""
import numpy as np
import pytest
import sympy as sp

from oracle import disk, grid, heat, ns, transforms as tr

xs, ys, zs = sp.symbols('x y z')


def _cyl_grid(p, m, n):
    TH, RR, ZZ = np.meshgrid(grid.theta_points(p), grid.cheb_points(m), grid.cheb_points(n), indexing='ij')
    return TH, RR, ZZ


def _vals(expr, p, m, n):
    TH, RR, ZZ = _cyl_grid(p, m, n)
    f = sp.lambdify((xs, ys, zs), expr, 'numpy')
    return f(RR * np.cos(TH), RR * np.sin(TH), ZZ) + 0.0 * RR


def _curl(F):
    Fx, Fy, Fz = F
    return (sp.diff(Fz, ys) - sp.diff(Fy, zs), sp.diff(Fx, zs) - sp.diff(Fz, xs), sp.diff(Fy, xs) - sp.diff(Fx, ys))


def _pt_cart(lam, gam):
    """curl(lam z) + curl curl(gam z) in Cartesian components."""
    a = _curl((0, 0, lam))
    b = _curl(_curl((0, 0, gam)))
    return tuple(sp.expand(a[i] + b[i]) for i in range(3))


def _to_cyl(F, p, m, n):
    """Grid values of the cylindrical components of a Cartesian field."""
    TH, _, _ = _cyl_grid(p, m, n)
    Fx, Fy, Fz = (_vals(c, p, m, n) for c in F)
    return (Fx * np.cos(TH) + Fy * np.sin(TH), -Fx * np.sin(TH) + Fy * np.cos(TH), Fz)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


P, M, N = 18, 16, 12          # even n_r; resolves the degree-7 products below exactly

LAM = 1 + xs * zs + ys ** 2 - 2 * xs * ys * zs + xs ** 3
GAM = (1 - xs ** 2 - ys ** 2) * (1 - zs ** 2) * (2 + xs - ys * zs + xs * ys)


def test_spectral_derivatives_on_a_polynomial():
    f = 3 + xs ** 2 * ys - ys * zs ** 3 + xs * ys * zs + ys ** 4
    C = tr.vals2coeffs(_vals(f, P, M, N))
    TH, RR, _ = _cyl_grid(P, M, N)
    fx, fy, fz = (_vals(sp.diff(f, v), P, M, N) for v in (xs, ys, zs))
    assert _rel(tr.coeffs2vals(ns.d_r(C)), np.cos(TH) * fx + np.sin(TH) * fy) < 1e-12
    assert _rel(tr.coeffs2vals(ns.d_theta(C)), RR * (-np.sin(TH) * fx + np.cos(TH) * fy)) < 1e-12
    assert _rel(tr.coeffs2vals(ns.d_z(C)), fz) < 1e-12


def test_pt_components_match_cartesian_curls():
    lam = tr.vals2coeffs(_vals(LAM, P, M, N))
    gam = tr.vals2coeffs(_vals(GAM, P, M, N))
    got = ns.pt_components(lam, gam)
    want = _to_cyl(_pt_cart(LAM, GAM), P, M, N)
    for g, w in zip(got, want):
        assert _rel(g, w) < 1e-11


def test_ptpoisson_right_sides_of_curl_n():
    Nc = (xs * ys * zs + ys ** 2, 1 - xs * zs ** 2 + xs * ys, xs ** 2 - ys * zs + xs * ys * zs)
    a = _curl(Nc)
    s1_want = _vals(a[2], P, M, N)
    s2_want = _vals(_curl(a)[2], P, M, N)
    s1, s2 = ns.curl_pt_rhs(_to_cyl(Nc, P, M, N))
    assert _rel(tr.coeffs2vals(s1), s1_want) < 1e-11
    assert _rel(tr.coeffs2vals(s2), s2_want) < 1e-11


def test_nonlinear_term_of_a_manufactured_flow():
    """Velocity potentials (lambda_v, gamma_v) with gamma_v = 0 on the whole
    wall; the vorticity state follows from eq. ptcurl: lambda_w = -lap gamma_v,
    gamma_w = lambda_v.  The oracle recovers gamma_v by its Poisson solve and
    must reproduce z . curl(v x omega) and z . curl curl(v x omega)."""
    lam_v, gam_v = LAM, GAM
    lap = sp.diff(gam_v, xs, 2) + sp.diff(gam_v, ys, 2) + sp.diff(gam_v, zs, 2)
    lam_w, gam_w = sp.expand(-lap), lam_v
    v = _pt_cart(lam_v, gam_v)
    w = _pt_cart(lam_w, gam_w)
    assert all(sp.expand(a - b) == 0 for a, b in zip(_curl(v), w))       # omega = curl v: eq. ptcurl
    Nc = (v[1] * w[2] - v[2] * w[1], v[2] * w[0] - v[0] * w[2], v[0] * w[1] - v[1] * w[0])
    a = _curl(Nc)
    Lw = tr.vals2coeffs(_vals(lam_w, P, M, N))
    Gw = tr.vals2coeffs(_vals(gam_w, P, M, N))
    _, _, s1, s2 = ns.nonlinear_pt(Lw, Gw, return_rhs=True)
    assert _rel(tr.coeffs2vals(s1), _vals(a[2], P, M, N)) < 1e-10
    assert _rel(tr.coeffs2vals(s2), _vals(_curl(a)[2], P, M, N)) < 1e-10


def test_horizontal_solves_recover_the_potentials():
    """eq. ptpoisson: z . V = -Delta_h gamma and z . curl V = -Delta_h lambda;
    with potentials that vanish at r = 1 the two horizontal solves return
    them exactly (tau exactness)."""
    lam = (1 - xs ** 2 - ys ** 2) * (xs - ys * zs + 3 * zs ** 2)
    gam = GAM
    V = _pt_cart(lam, gam)
    zV = tr.vals2coeffs(_vals(V[2], P, M, N))
    zcV = tr.vals2coeffs(_vals(_curl(V)[2], P, M, N))
    assert _rel(disk.horizontal_poisson(zV), tr.vals2coeffs(_vals(gam, P, M, N))) < 1e-12
    assert _rel(disk.horizontal_poisson(zcV), tr.vals2coeffs(_vals(lam, P, M, N))) < 1e-12


def test_nonlinear_term_is_quadratic_and_step_has_the_linear_limit():
    rng = np.random.default_rng(3)
    from paper_2206_04827_gb300 import inputs
    p, m, n = 8, 12, 9
    Lw = inputs.smooth_coeffs(p, m, n, 1.4, rng)
    Gw = inputs.smooth_coeffs(p, m, n, 1.4, rng)
    a1, g1 = ns.nonlinear_pt(Lw, Gw)
    a2, g2 = ns.nonlinear_pt(2 * Lw, 2 * Gw)
    assert _rel(a2, 4 * a1) < 1e-12 and _rel(g2, 4 * g1) < 1e-12
    Re, dt, eps = 50.0, 1e-2, 1e-6
    l_eps, g_eps = ns.ns_steps(eps * Lw, eps * Gw, Re, dt, 2)
    l_lin = heat.heat_steps(Lw, np.zeros_like(Lw), 1.0 / Re, dt, 2)
    g_lin = heat.heat_steps(Gw, np.zeros_like(Gw), 1.0 / Re, dt, 2)
    assert _rel(l_eps / eps, l_lin) < 1e-4 and _rel(g_eps / eps, g_lin) < 1e-4
    assert _rel(l_eps / eps, l_lin) > 0.0                                # the nonlinear term is present


def test_odd_radial_grids_are_rejected():
    with pytest.raises(ValueError):
        ns.pt_components(np.zeros((4, 9, 5)), np.zeros((4, 9, 5)))


EXT_BITS = np.finfo(np.longdouble).nmant
needs_ext = pytest.mark.skipif(EXT_BITS < 63, reason='np.longdouble is not wider than double here')


@needs_ext
def test_extended_transforms_match_and_round_trip():
    x = np.random.default_rng(11).standard_normal((10, 12, 9))
    c = tr.vals2coeffs_ext(x.astype(tr.EXT))
    assert _rel(np.asarray(c, dtype=np.float64), tr.vals2coeffs(x)) < 1e-15
    assert np.abs(tr.coeffs2vals_ext(c) - x).max() < 1e-17 * np.abs(x).max()


def test_exact_derivative_matrix():
    M = ns.cheb_derivative_matrix_ext(9)
    assert M[0, 3] == 3 and M[2, 3] == 6 and M[1, 3] == 0                 # T_3' = 12 x^2 - 3 = 6 T_2 + 3 T_0
    assert M[1, 4] == 8 and M[3, 4] == 8 and M[0, 4] == 0                 # T_4' = 32 x^3 - 16 x = 8 T_3 + 8 T_1
    C = np.eye(9)[None]                                                   # the FP64 matrix (D1, then C01 solve)
    assert _rel(np.asarray(M, dtype=np.float64), ns.d_axis(C, 1)[0]) < 1e-14


@needs_ext
def test_extended_nonlinear_term_of_the_manufactured_flow():
    lam_v, gam_v = LAM, GAM
    lap = sp.diff(gam_v, xs, 2) + sp.diff(gam_v, ys, 2) + sp.diff(gam_v, zs, 2)
    lam_w, gam_w = sp.expand(-lap), lam_v
    v = _pt_cart(lam_v, gam_v)
    w = _pt_cart(lam_w, gam_w)
    Nc = (v[1] * w[2] - v[2] * w[1], v[2] * w[0] - v[0] * w[2], v[0] * w[1] - v[1] * w[0])
    a = _curl(Nc)
    Lw = tr.vals2coeffs(_vals(lam_w, P, M, N))
    Gw = tr.vals2coeffs(_vals(gam_w, P, M, N))
    # the same formulas as the FP64 path (the bar is set by the FP64 rounding of the input coefficients,
    # which the derivatives amplify; the building blocks' own accuracy is pinned above)
    _, _, s1, s2 = ns.nonlinear_pt(Lw, Gw, return_rhs=True, extended=True)
    assert _rel(tr.coeffs2vals(s1), _vals(a[2], P, M, N)) < 1e-10
    assert _rel(tr.coeffs2vals(s2), _vals(_curl(a)[2], P, M, N)) < 1e-10


@needs_ext
def test_extended_step_agrees_with_the_fp64_step():
    from paper_2206_04827_gb300 import inputs
    rng = np.random.default_rng(5)
    Lw = 3.0 * inputs.smooth_coeffs(8, 12, 11, 1.4, rng)
    Gw = 3.0 * inputs.smooth_coeffs(8, 12, 11, 1.4, rng)
    l64, g64 = ns.ns_steps(Lw, Gw, 20.0, 5e-3, 2)
    lx, gx = ns.ns_steps(Lw, Gw, 20.0, 5e-3, 2, extended=True)
    assert _rel(lx, l64) < 1e-12 and _rel(gx, g64) < 1e-12
