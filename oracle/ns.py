"""Navier-Stokes time step in poloidal-toroidal form (oracle; test
infrastructure only).

Section 4, eq. ns: (d_t - Re^-1 lap) omega = curl(v x omega), omega = curl v.
The state is the PT decomposition (eq. pt) of the vorticity,
omega = curl(lambda_w z) + curl curl(gamma_w z), as half-complex CCF
coefficient arrays [p][m][n] (see ``transforms``).  One step, in the order
of Section 4:

1. velocity potentials from eq. ptcurl with W = omega, V = v:
   lambda_v = gamma_w  and  -lap gamma_v = lambda_w  (one Poisson solve);
2. cylindrical components of v and omega in value space from eq. pt:
   V_r = r^-1 d_th lambda + d_r d_z gamma,
   V_th = -d_r lambda + r^-1 d_th d_z gamma,
   V_z = -Delta_h gamma,  Delta_h = d_r^2 + r^-1 d_r + r^-2 d_th^2;
3. the nonlinear term N = v x omega pointwise on the grid (pseudo-spectral);
4. the PT decomposition (lambda_a, gamma_a) of a = curl N from eq. ptpoisson:
   -Delta_h gamma_a = z . a = d_r N_th + N_th / r - r^-1 d_th N_r,
   -Delta_h lambda_a = z . curl a = d_z (d_r N_r + N_r / r + r^-1 d_th N_th) - Delta_h N_z
   (two horizontal Poisson solves);
5. eq. NSrewrite by the first-order implicit-explicit BDF (the IMEX family
   the paper cites): the diffusion implicit, the nonlinear term explicit,
   (1 - dt Re^-1 lap) lambda_w^{n+1} = lambda_w^n + dt lambda_a^n and the
   same for gamma_w: two BDF1 heat steps with alpha = 1/Re and forcing
   (lambda_a, gamma_a).

Derivatives are taken on coefficients (d_r, d_z: the Chebyshev derivative as
D1 of Section 3 followed by the U -> T conversion, i.e. solving with C01;
d_th: multiplication by i w on the half-complex slices, zero on the Nyquist
slice, whose derivative vanishes on the grid); products and the factors 1/r
are applied to grid values, which needs an even n_r (no grid point at r = 0).

Reading of the boundary conditions (the appendix's no-slip conditions -- the
vector-potential conditions and Quartapelle's integral conditions with a
low-rank update -- are not specified to the point of an implementation):
every scalar solve above takes the homogeneous Dirichlet data the rest of the
solver uses: gamma_v = 0 on the whole wall, gamma_a = lambda_a = 0 at
r = +-1 (horizontal solves have no z condition), lambda_w = gamma_w = 0 on
the whole wall.
"""
import numpy as np

from . import grid, heat, operators as ops
from .disk import horizontal_poisson
from .transforms import coeffs2vals, vals2coeffs


def d_axis(C, axis):
    """d/dx of a Chebyshev T-series along `axis` (1 = r, 2 = z): the T -> U
    derivative D1 of Section 3, then back to T coefficients through C01."""
    L = C.shape[axis]
    M = np.linalg.solve(ops.conv_T_to_U(L), ops.diff1_T_to_U(L))    # T -> T derivative matrix
    return np.moveaxis(np.tensordot(M, np.moveaxis(C, axis, 0), axes=(1, 0)), 0, axis)


def d_r(C):
    return d_axis(C, 1)


def d_z(C):
    return d_axis(C, 2)


def d_theta(C):
    """d/dtheta on half-complex slices: c_w e^{i w theta} -> i w c_w e^{i w theta}
    (slice 2w-1 = Re, 2w = Im); zero on slice 0 and on the Nyquist slice."""
    p = C.shape[0]
    D = np.zeros_like(C)
    for w in range(1, p // 2):
        D[2 * w - 1] = -w * C[2 * w]
        D[2 * w] = w * C[2 * w - 1]
    return D


def _radius(m):
    if m % 2:
        raise ValueError('the pseudo-spectral step needs an even n_r (no grid point at r = 0)')
    return grid.cheb_points(m)[None, :, None]


def pt_components(lam, gam):
    """Grid values (V_r, V_th, V_z) of V = curl(lam z) + curl curl(gam z) (eq. pt)."""
    r = _radius(lam.shape[1])
    v = coeffs2vals
    Vr = v(d_theta(lam)) / r + v(d_r(d_z(gam)))
    Vth = -v(d_r(lam)) + v(d_theta(d_z(gam))) / r
    Vz = -(v(d_r(d_r(gam))) + v(d_r(gam)) / r + v(d_theta(d_theta(gam))) / r ** 2)
    return Vr, Vth, Vz


def cross(a, b):
    """Pointwise cylindrical cross product a x b of component triples."""
    ar, at, az = a
    br, bt, bz = b
    return at * bz - az * bt, az * br - ar * bz, ar * bt - at * br


def curl_pt_rhs(N):
    """Right sides of eq. ptpoisson for a = curl N, as coefficients:
    s1 = z . curl N, s2 = z . curl curl N (N given by grid values)."""
    Nr, Nt, Nz = N
    r = _radius(Nr.shape[1])
    v, c = coeffs2vals, vals2coeffs
    Cr, Ct, Cz = c(Nr), c(Nt), c(Nz)
    s1 = v(d_r(Ct)) + Nt / r - v(d_theta(Cr)) / r
    div_h = c(v(d_r(Cr)) + Nr / r + v(d_theta(Ct)) / r)
    lap_h_Nz = v(d_r(d_r(Cz))) + v(d_r(Cz)) / r + v(d_theta(d_theta(Cz))) / r ** 2
    s2 = v(d_z(div_h)) - lap_h_Nz
    return c(s1), c(s2)


def nonlinear_pt(lam_w, gam_w, return_rhs=False):
    """(lambda_a, gamma_a): the PT decomposition of a = curl(v x omega) for the
    vorticity state (lam_w, gam_w) -- steps 1 to 4 of the module docstring
    (with return_rhs also the coefficients of s1 = z . a and s2 = z . curl a)."""
    lam_v, gam_v = gam_w.copy(), heat.poisson(lam_w)
    N = cross(pt_components(lam_v, gam_v), pt_components(lam_w, gam_w))
    s1, s2 = curl_pt_rhs(N)
    out = (horizontal_poisson(s2), horizontal_poisson(s1))
    return out + (s1, s2) if return_rhs else out


def ns_steps(lam_w, gam_w, Re, dt, nsteps):
    """nsteps IMEX BDF1 steps of eq. NSrewrite (step 5 of the module docstring)."""
    lam_w = np.array(lam_w, dtype=np.float64, copy=True)
    gam_w = np.array(gam_w, dtype=np.float64, copy=True)
    for _ in range(nsteps):
        lam_a, gam_a = nonlinear_pt(lam_w, gam_w)
        lam_w = heat.heat_steps(lam_w, lam_a, 1.0 / Re, dt, 1)
        gam_w = heat.heat_steps(gam_w, gam_a, 1.0 / Re, dt, 1)
    return lam_w, gam_w
