"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the solver: it draws random numbers and
evaluates closed-form fields at coordinates that the caller passes in (each
side of a comparison brings its own grid).  Nothing here transforms, solves
or steps.

Workloads (the paper's Table 1 problems are not specified, so these follow
the problem statement of Section 3 with synthetic data):

* ``smooth_coeffs``    -- half-complex CCF coefficient array with entries
                          N(0,1) * decay^-(i + j + |k|), zero where the radial
                          degree i and the wavenumber k differ in parity (the
                          coefficients of a real field on the doubled grid),
                          zero on the Nyquist slice.
* ``eigenmode_values`` -- sum of Bessel x sine eigenmodes
                          J_mu(j_{mu,nu} r) {cos, sin}(mu theta) sin(nu pi (z+1)/2)
                          of the Dirichlet Laplacian on the cylinder.
* ``manufactured_u`` / ``manufactured_f`` -- u = (1-r^2)(1-z^2) exp(r cos th + z/2)
                          and f = -lap u in closed form.
"""
import numpy as np
from scipy import special


def rng_for(seed):
    return np.random.default_rng(seed)


def smooth_coeffs(p, m, n, decay, rng):
    """Half-complex coefficients [p][m][n] of a smooth real field (layout:
    slice 0 = k 0, slices 2k-1 / 2k = Re / Im of k, slice p-1 = Nyquist)."""
    out = np.zeros((p, m, n))
    i = np.arange(m)[:, None]
    j = np.arange(n)[None, :]
    for s in range(p - 1):
        k = 0 if s == 0 else (s + 1) // 2
        a = rng.standard_normal((m, n)) * float(decay) ** (-(i + j + k))
        a[np.broadcast_to((i % 2) != (k % 2), (m, n))] = 0.0
        out[s] = a
    return out


def eigenmode_list(count, rng, max_mu=6, max_nu=4):
    """Draw `count` distinct (mu, nu, trig) eigenmodes with N(0,1) amplitudes.
    trig = 0 selects cos(mu theta), 1 selects sin(mu theta) (not for mu = 0)."""
    pool = [(mu, nu, t) for mu in range(max_mu + 1) for nu in range(1, max_nu + 1)
            for t in ((0,) if mu == 0 else (0, 1))]
    idx = rng.choice(len(pool), size=count, replace=False)
    amps = rng.standard_normal(count)
    return [(pool[q][0], pool[q][1], pool[q][2], float(a)) for q, a in zip(idx, amps)]


def bessel_zero(mu, nu):
    """nu-th positive zero j_{mu,nu} of J_mu."""
    return float(special.jn_zeros(mu, nu)[-1])


def eigenvalue(mu, nu):
    """Dirichlet Laplacian eigenvalue j_{mu,nu}^2 + (nu pi / 2)^2 of the mode."""
    return bessel_zero(mu, nu) ** 2 + (nu * np.pi / 2.0) ** 2


def eigenmode_values(r, z, theta, modes):
    """Sum of eigenmodes on the tensor grid; returns [p][m][n] = [theta][r][z]."""
    TH, RR, ZZ = np.meshgrid(np.asarray(theta), np.asarray(r), np.asarray(z), indexing='ij')
    out = np.zeros(TH.shape)
    for mu, nu, t, a in modes:
        ang = np.cos(mu * TH) if t == 0 else np.sin(mu * TH)
        out += a * special.jv(mu, bessel_zero(mu, nu) * RR) * ang * np.sin(nu * np.pi * (ZZ + 1.0) / 2.0)
    return out


def manufactured_u(r, z, theta):
    """u = (1 - r^2)(1 - z^2) exp(r cos theta + z/2) on the tensor grid."""
    TH, RR, ZZ = np.meshgrid(np.asarray(theta), np.asarray(r), np.asarray(z), indexing='ij')
    return (1.0 - RR ** 2) * (1.0 - ZZ ** 2) * np.exp(RR * np.cos(TH) + 0.5 * ZZ)


def manufactured_f(r, z, theta):
    """f = -lap u for ``manufactured_u``:
    f = -(z + 1)((5z + 3) r^2 + 16 (z - 1) r cos theta + 11 z - 19) exp(r cos theta + z/2) / 4."""
    TH, RR, ZZ = np.meshgrid(np.asarray(theta), np.asarray(r), np.asarray(z), indexing='ij')
    x = RR * np.cos(TH)
    return -(ZZ + 1.0) * ((5.0 * ZZ + 3.0) * RR ** 2 + 16.0 * (ZZ - 1.0) * x + 11.0 * ZZ - 19.0) \
        * np.exp(x + 0.5 * ZZ) / 4.0
