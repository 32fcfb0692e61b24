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

Extended precision (``extended=True``): the nonlinear term differentiates
the state up to four times and takes products on the grid, so FP64 rounding
of order eps * max|values| in its intermediate arrays reaches the low-order
coefficients of lambda_a amplified (at 128^3 with the smooth seeded states
of the workloads, a plain FP64 evaluation of one step ends ~4e-11 from the
exact result).  The extended path evaluates steps 2 to 4 in np.longdouble
(transforms by their direct sums, the exact Chebyshev derivative matrix),
with the Poisson solve of step 1 and the heat steps of step 5 refined
(``heat._solve``); it writes reference values, and the FP64 path is the
oracle of every other check.

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
from . import transforms as otr
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


def cheb_derivative_matrix_ext(L):
    """T -> T derivative matrix in extended precision from its closed form:
    T_j' = 2j sum over k < j with j - k odd of T_k, the k = 0 term halved."""
    M = np.zeros((L, L), dtype=otr.EXT)
    for j in range(1, L):
        for k in range(j - 1, -1, -2):
            M[k, j] = otr.EXT(2 * j) / (2 if k == 0 else 1)
    return M


def d_axis_ext(C, axis):
    M = cheb_derivative_matrix_ext(C.shape[axis])
    return np.moveaxis(np.tensordot(M, np.moveaxis(C, axis, 0), axes=(1, 0)), 0, axis)


class _Arith:
    """The value-space arithmetic of steps 2 to 4: FP64 or extended."""

    def __init__(self, extended):
        self.ext = extended
        self.v = otr.coeffs2vals_ext if extended else coeffs2vals
        self.c = otr.vals2coeffs_ext if extended else vals2coeffs
        self.d_r = (lambda C: d_axis_ext(C, 1)) if extended else d_r
        self.d_z = (lambda C: d_axis_ext(C, 2)) if extended else d_z

    def radius(self, m):
        if m % 2:
            raise ValueError('the pseudo-spectral step needs an even n_r (no grid point at r = 0)')
        if self.ext:
            return otr._cheb_at_grid_ext(m)[:, 1][None, :, None]       # T_1(x_a) = x_a
        return grid.cheb_points(m)[None, :, None]


FP64, EXTENDED = _Arith(False), _Arith(True)


def d_theta(C):
    """d/dtheta on half-complex slices: c_w e^{i w theta} -> i w c_w e^{i w theta}
    (slice 2w-1 = Re, 2w = Im); zero on slice 0 and on the Nyquist slice."""
    p = C.shape[0]
    D = np.zeros_like(C)
    for w in range(1, p // 2):
        D[2 * w - 1] = -w * C[2 * w]
        D[2 * w] = w * C[2 * w - 1]
    return D


def pt_components(lam, gam, ar=FP64):
    """Grid values (V_r, V_th, V_z) of V = curl(lam z) + curl curl(gam z) (eq. pt)."""
    r = ar.radius(lam.shape[1])
    v, d_r, d_z = ar.v, ar.d_r, ar.d_z
    Vr = v(d_theta(lam)) / r + v(d_r(d_z(gam)))
    Vth = -v(d_r(lam)) + v(d_theta(d_z(gam))) / r
    Vz = -(v(d_r(d_r(gam))) + v(d_r(gam)) / r + v(d_theta(d_theta(gam))) / r ** 2)
    return Vr, Vth, Vz


def cross(a, b):
    """Pointwise cylindrical cross product a x b of component triples."""
    ar, at, az = a
    br, bt, bz = b
    return at * bz - az * bt, az * br - ar * bz, ar * bt - at * br


def curl_pt_rhs(N, ar=FP64):
    """Right sides of eq. ptpoisson for a = curl N, as coefficients:
    s1 = z . curl N, s2 = z . curl curl N (N given by grid values)."""
    Nr, Nt, Nz = N
    r = ar.radius(Nr.shape[1])
    v, c, d_r, d_z = ar.v, ar.c, ar.d_r, ar.d_z
    Cr, Ct, Cz = c(Nr), c(Nt), c(Nz)
    s1 = v(d_r(Ct)) + Nt / r - v(d_theta(Cr)) / r
    div_h = c(v(d_r(Cr)) + Nr / r + v(d_theta(Ct)) / r)
    lap_h_Nz = v(d_r(d_r(Cz))) + v(d_r(Cz)) / r + v(d_theta(d_theta(Cz))) / r ** 2
    s2 = v(d_z(div_h)) - lap_h_Nz
    return c(s1), c(s2)


def nonlinear_pt(lam_w, gam_w, return_rhs=False, extended=False):
    """(lambda_a, gamma_a): the PT decomposition of a = curl(v x omega) for the
    vorticity state (lam_w, gam_w) -- steps 1 to 4 of the module docstring
    (with return_rhs also the coefficients of s1 = z . a and s2 = z . curl a).
    extended: steps 2 to 4 in extended precision, step 1 refined."""
    ar = EXTENDED if extended else FP64
    gam_v = heat.poisson(lam_w, refine=2 if extended else 0)
    if extended:
        lam_v, gam_v = gam_w.astype(otr.EXT), gam_v.astype(otr.EXT)
        lam_w, gam_w = lam_w.astype(otr.EXT), gam_w.astype(otr.EXT)
    else:
        lam_v = gam_w.copy()
    N = cross(pt_components(lam_v, gam_v, ar), pt_components(lam_w, gam_w, ar))
    s1, s2 = (np.asarray(x, dtype=np.float64) for x in curl_pt_rhs(N, ar))
    out = (horizontal_poisson(s2), horizontal_poisson(s1))
    return out + (s1, s2) if return_rhs else out


def ns_steps(lam_w, gam_w, Re, dt, nsteps, extended=False):
    """nsteps IMEX BDF1 steps of eq. NSrewrite (step 5 of the module docstring);
    extended: the nonlinear term in extended precision and refined solves."""
    lam_w = np.array(lam_w, dtype=np.float64, copy=True)
    gam_w = np.array(gam_w, dtype=np.float64, copy=True)
    refine = 2 if extended else 0
    for _ in range(nsteps):
        lam_a, gam_a = nonlinear_pt(lam_w, gam_w, extended=extended)
        lam_w = heat.heat_steps(lam_w, lam_a, 1.0 / Re, dt, 1, refine=refine)
        gam_w = heat.heat_steps(gam_w, gam_a, 1.0 / Re, dt, 1, refine=refine)
    return lam_w, gam_w
