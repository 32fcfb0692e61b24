"""Poisson solve, BDF1 heat stepping and its discrete adjoint (oracle; test infrastructure only).

All arrays are half-complex coefficient arrays [p][m][n] (see ``transforms``).
Each half-complex slice is a real slice of one wavenumber |k|; the operators
are real and depend on k^2 only (eq. HelmholtzMatEqn), so every slice is an
independent real matrix equation ("decouple in theta", Section 3).

* ``poisson``     -- -lap u = f with zero Dirichlet data (Section 4 Poisson
                     solves; Section 3 machinery without the identity term).
* ``heat_steps``  -- BDF1 (Section 3, BDF 1: kappa = h, delta X = X_n) with the
                     forcing of step n -> n+1 taken at level n (the
                     extrapolation g(t+h) ~ g(t) stated beside eq.
                     HelmholtzMatEqn).
* ``bdf_coefficients`` / ``heat_bdf`` -- the b-th order BDF of Section 3
                     (BDF 4 printed; delta^(b) defined by sampling at t, t-h,
                     ... and taking differences): kappa^(b) and delta^(b) from
                     the backward-difference form, the first steps of a run
                     through lower orders while fewer than b past states are
                     known (reading: start-up is unstated).
* ``heat_adjoint``-- gradients of a scalar loss of X_N with respect to X_0,
                     every g_n and alpha, by the chain rule through the
                     direct solves (no part of the paper; the transpose of
                     the stepping map above).
"""
from fractions import Fraction
from math import comb

import numpy as np

from .sylvester import ModeSystem, BartelsStewart, bordered_solve, solve_kron
from .transforms import slice_wavenumber


class _systems(dict):
    """One ModeSystem and direct solver per distinct |k| (slices share them),
    built on first use."""

    def __init__(self, m, n, p, kind, kappa_alpha=None):
        super().__init__()
        self.args = (m, n, kind, kappa_alpha)

    def __missing__(self, k):
        m, n, kind, ka = self.args
        ms = ModeSystem(m, n, k, kind, ka)
        self[k] = (ms, BartelsStewart(ms.A, ms.B, ms.C, ms.D))
        return self[k]


def _solve(ms, bs, E, brute, refine):
    """Y with A Y B^T + C Y D^T = E: QZ Bartels-Stewart (or the dense Kronecker
    solve when brute), then `refine` steps of iterative refinement whose
    residual E - (A Y B^T + C Y D^T) is formed in extended precision
    (np.longdouble).  Refinement is not part of the paper: a textbook remedy
    for the forward error of the direct solve on large grids (about 1e-11 at
    512 x 512 for the heat system), used to write stored reference values."""
    Y = solve_kron(ms.A, ms.B, ms.C, ms.D, E) if brute else bs.solve(E)
    if refine:
        L = np.longdouble
        A, B, C, D = (x.astype(L) for x in (ms.A, ms.B, ms.C, ms.D))
        for _ in range(refine):
            Yl = Y.astype(L)
            R = E.astype(L) - (A @ Yl @ B.T + C @ Yl @ D.T)
            Y = Y + bs.solve(np.asarray(R, dtype=np.float64))
    return Y


def lifting(bc_vals):
    """Coefficients of the transfinite (Gordon-Hall) blend of the boundary
    values of bc_vals ([p][m][n] grid values; only the nodes with j in
    {0, m-1} or k in {0, n-1} are read): linear in r between the faces
    r = -1, +1 plus linear in z between z = -1, +1 minus the bilinear corner
    term.  Its traces on the four faces are the data's interpolants (reading
    of the unstated boundary conditions: Dirichlet data by lifting)."""
    from .grid import cheb_points
    from .transforms import vals2coeffs
    b = np.asarray(bc_vals, dtype=np.float64)
    p, m, n = b.shape
    r = cheb_points(m)[None, :, None]
    z = cheb_points(n)[None, None, :]
    lo_r, hi_r = b[:, :1, :], b[:, -1:, :]
    lo_z, hi_z = b[:, :, :1], b[:, :, -1:]
    Pr = 0.5 * (1 - r) * lo_r + 0.5 * (1 + r) * hi_r
    Pz = 0.5 * (1 - z) * lo_z + 0.5 * (1 + z) * hi_z
    PrPz = (0.25 * (1 - r) * (1 - z) * b[:, :1, :1] + 0.25 * (1 - r) * (1 + z) * b[:, :1, -1:]
            + 0.25 * (1 + r) * (1 - z) * b[:, -1:, :1] + 0.25 * (1 + r) * (1 + z) * b[:, -1:, -1:])
    return vals2coeffs(Pr + Pz - PrPz)


def poisson(F, slices=None, brute=False, bc=None, refine=0):
    """Coefficients u of -lap u = f for half-complex coefficients F of f.

    bc: optional [p][m][n] grid values whose boundary nodes hold the Dirichlet
    data (consistent at the corners); u = u0 + W with W = lifting(bc) and u0
    the zero-data solution of the equation with right side corrected by the
    operator applied to W.  brute=True solves the bordered tau system
    (boundary rows appended) by dense least squares instead."""
    p, m, n = F.shape
    sys_ = _systems(m, n, p, 'poisson')
    U = np.zeros_like(F)
    W = lifting(bc) if bc is not None else np.zeros_like(F)
    for s in (range(p) if slices is None else slices):
        k = slice_wavenumber(s, p)
        ms, bs = sys_[k]
        if brute and bc is not None:
            U[s] = bordered_solve(m, n, k, 'poisson', None, F[s], W[s])
            continue
        E = ms.rhs(F[s]) - ms.full_apply(W[s])
        Y = _solve(ms, bs, E, brute, refine)
        U[s] = ms.expand(Y) + W[s]
    return U


def heat_steps(X0, g, alpha, dt, nsteps, slices=None, brute=False, return_all=False, bc=None, refine=0):
    """BDF1: X_{n+1} solves eq. HelmholtzMatEqn with delta X = X_n, kappa = dt.

    g is either one coefficient array (constant forcing) or an array of
    shape [nsteps][p][m][n] (g[n] is used by the step n -> n+1).  bc:
    optional time-constant Dirichlet data as in ``poisson`` (X_{n+1} = S Y S^T
    + W, the right side corrected by the step operator applied to W).  refine:
    steps of iterative refinement per solve (see ``_solve``)."""
    p, m, n = X0.shape
    kappa = dt
    sys_ = _systems(m, n, p, 'heat', kappa * alpha)
    W = lifting(bc) if bc is not None else None
    g = np.asarray(g, dtype=np.float64)
    X = np.array(X0, dtype=np.float64, copy=True)
    traj = [X.copy()] if return_all else None
    todo = range(p) if slices is None else slices
    for step in range(nsteps):
        gn = g[step] if g.ndim == 4 else g
        Xn = np.zeros_like(X)
        for s in todo:
            k = slice_wavenumber(s, p)
            ms, bs = sys_[k]
            if W is not None and brute:
                Xn[s] = bordered_solve(m, n, k, 'heat', kappa * alpha, X[s] + kappa * gn[s], W[s])
                continue
            E = ms.rhs(X[s] + kappa * gn[s])
            if W is not None:
                E = E - ms.full_apply(W[s])
            Y = _solve(ms, bs, E, brute, refine)
            Xn[s] = ms.expand(Y) + (W[s] if W is not None else 0.0)
        X = Xn
        if return_all:
            traj.append(X.copy())
    return (X, traj) if return_all else X


def bdf_coefficients(b):
    """(kappa^(b) / h, [beta_0 .. beta_{b-1}]) as exact fractions for the
    b-th order BDF  y_{n+1} - kappa y'_{n+1} = sum_i beta_i y_{n-i}.

    Definition used: the backward-difference form sum_{j=1..b} (1/j) nabla^j
    y_{n+1} = h y'_{n+1} with nabla y_{n+1} = y_{n+1} - y_n (the differences of
    the samples at t+h, t, t-h, ...), divided by its coefficient of y_{n+1}."""
    if not 1 <= b <= 6:
        raise ValueError('BDF order must be 1..6')
    # coefficient of y_{n+1-i} in sum_j (1/j) nabla^j y_{n+1}
    a = [sum(Fraction((-1) ** i * comb(j, i), j) for j in range(max(i, 1), b + 1)) for i in range(b + 1)]
    return 1 / a[0], [-a[i] / a[0] for i in range(1, b + 1)]


def heat_bdf(hist, g, alpha, dt, order, nsteps, nvalid=None, slices=None, brute=False, bc=None,
             return_all=False):
    """The b-th order BDF run (b = order) of eq. HelmholtzMatEqn:
    (R_2 - kappa alpha L) X_{n+1} C02^T - kappa alpha R_2 X_{n+1} D2^T
        = R_2 (delta^(b) X_n + kappa g_n) C02^T,
    kappa = kappa^(b), delta^(b) X_n = sum_i beta_i X_{n-i}.

    hist: [order][p][m][n] with hist[i] = X_{n-i}; only the first nvalid
    (default: order) are known.  A step with v known states uses BDF min(order,
    v).  g: one array or [nsteps][p][m][n] (g[s] drives step s).  bc: Dirichlet
    data as in ``poisson`` (lifting per step with that step's operator).
    Returns the new history (slot i = X_{n+nsteps-i}; slots beyond the known
    states are zero), plus the list of all new states when return_all."""
    hist = np.array(hist, dtype=np.float64, copy=True)
    order = int(order)
    _, p, m, n = hist.shape
    v = order if nvalid is None else int(nvalid)
    known = [hist[i] for i in range(v)]                # newest first
    g = np.asarray(g, dtype=np.float64)
    W = lifting(bc) if bc is not None else None
    todo = range(p) if slices is None else slices
    systems = {}
    new = []
    for step in range(nsteps):
        b = min(order, len(known))
        kap, beta = bdf_coefficients(b)
        kappa = float(kap) * dt
        if b not in systems:
            systems[b] = _systems(m, n, p, 'heat', kappa * alpha)
        sys_ = systems[b]
        gn = g[step] if g.ndim == 4 else g
        delta = sum(float(beta[i]) * known[i] for i in range(b))
        Xn = np.zeros((p, m, n))
        for s in todo:
            k = slice_wavenumber(s, p)
            ms, bs = sys_[k]
            if W is not None and brute:
                Xn[s] = bordered_solve(m, n, k, 'heat', kappa * alpha, delta[s] + kappa * gn[s], W[s])
                continue
            E = ms.rhs(delta[s] + kappa * gn[s])
            if W is not None:
                E = E - ms.full_apply(W[s])
            Y = solve_kron(ms.A, ms.B, ms.C, ms.D, E) if brute else bs.solve(E)
            Xn[s] = ms.expand(Y) + (W[s] if W is not None else 0.0)
        known = [Xn] + known[:order - 1]
        new.append(Xn)
    out = np.zeros_like(hist)
    for i, X in enumerate(known):
        out[i] = X
    return (out, new) if return_all else out


def heat_bdf_adjoint(hist, g, alpha, dt, order, nsteps, dL_dhistN, nvalid=None, slices=None, bc=None):
    """Reverse-mode derivatives of L(final history) for ``heat_bdf``.

    Returns (dL/dhist0, dL/dg, dL/dalpha): dL/dhist0 is [order][p][m][n] with
    slot i = dL/dX_{-i} (zero beyond the known states), dL/dg has the shape of
    g.  Step s (order b, kappa = kappa^(b) h): E = Rhs(sum_i beta_i X_{s-i} +
    kappa g_s), Y = Sylv^-1 E, X_{s+1} = S Y S^T (+ W).  Reverse: lam_j =
    dL/dX_j accumulated; mu = S^T lam_{s+1} S; Lam = Sylv^-T mu; w = Rhs^T Lam;
    lam_{s-i} += beta_i w; dL/dg_s = kappa w; dL/dalpha -= <Lam, dSylv/dalpha Y>
    (+ the derivative of the lifted right side, as in ``heat_adjoint``)."""
    hist = np.asarray(hist, dtype=np.float64)
    order = int(order)
    _, p, m, n = hist.shape
    v0 = order if nvalid is None else int(nvalid)
    g = np.asarray(g, dtype=np.float64)
    const_g = g.ndim == 3
    W = lifting(bc) if bc is not None else np.zeros((p, m, n))
    _, new = heat_bdf(hist, g, alpha, dt, order, nsteps, nvalid=v0, slices=slices, bc=bc, return_all=True)
    # states by time index j = -(v0-1) .. nsteps
    X = {-i: hist[i] for i in range(v0)}
    for s, Xs in enumerate(new):
        X[s + 1] = Xs
    lam = {j: np.zeros((p, m, n)) for j in X}
    for i in range(min(order, v0 + nsteps)):
        lam[nsteps - i] = lam[nsteps - i] + dL_dhistN[i]
    todo = range(p) if slices is None else slices
    dg = np.zeros_like(g)
    dalpha = 0.0
    systems = {}
    for s in reversed(range(nsteps)):
        b = min(order, v0 + s)
        kap, beta = bdf_coefficients(b)
        kappa = float(kap) * dt
        if b not in systems:
            systems[b] = _systems(m, n, p, 'heat', kappa * alpha)
        sys_ = systems[b]
        for sl in todo:
            ms, bs = sys_[slice_wavenumber(sl, p)]
            mu = ms.expand_T(lam[s + 1][sl])
            Lam = bs.solve_T(mu)
            w = ms.rhs_T(Lam)
            for i in range(b):
                lam[s - i][sl] += float(beta[i]) * w
            if const_g:
                dg[sl] += kappa * w
            else:
                dg[s, sl] = kappa * w
            Y = np.linalg.lstsq(ms.Sr, np.linalg.lstsq(ms.Sz, (X[s + 1][sl] - W[sl]).T, rcond=None)[0].T,
                                rcond=None)[0]
            dS = kappa * (ms.dA @ Y @ ms.B.T + ms.C @ Y @ ms.dD.T)
            if bc is not None:
                dS = dS + kappa * ms.full_apply_dka(W[sl])
            dalpha -= float(np.sum(Lam * dS))
    out = np.zeros_like(hist)
    for i in range(v0):
        out[i] = lam[-i]
    return out, dg, dalpha


def heat_adjoint(X0, g, alpha, dt, nsteps, dL_dXN, slices=None, bc=None):
    """Reverse-mode derivatives of L(X_N) for the BDF1 stepping above.

    Returns (dL/dX0, dL/dg, dL/dalpha); dL/dg has the shape of g (summed over
    the steps when g is one constant array).  With ``slices`` only those
    half-complex slices are processed (slices are independent), and dL/dalpha
    holds their contribution only.

    Step map per slice: E = Rhs(X_n + kappa g_n), Y = Sylv^-1 E, X_{n+1} = S Y S^T,
    with Sylv(Y) = A Y B^T + C Y D^T, A = C - kappa alpha Lr, D = -kappa alpha D2z.
    Reverse: mu = S^T lam S; Lam = Sylv^-T mu; lam_n = Rhs^T Lam;
    dL/dg_n = kappa lam_n; dL/dalpha += -<Lam, dSylv/dalpha Y_{n+1}>,
    dSylv/dalpha Y = kappa (dA Y B^T + C Y dD^T).

    bc: Dirichlet data as in ``heat_steps``.  Then X_{n+1} = S Y S^T + W and
    the right side carries -Full(W) (Full = the left operator on a full
    block), so dL/dalpha gains -<Lam, kappa dFull/d(kappa alpha) W> and Y is
    recovered from X_{n+1} - W; the other derivatives are unchanged (the data
    enter affinely)."""
    p, m, n = X0.shape
    kappa = dt
    sys_ = _systems(m, n, p, 'heat', kappa * alpha)
    g = np.asarray(g, dtype=np.float64)
    const_g = g.ndim == 3
    _, traj = heat_steps(X0, g, alpha, dt, nsteps, slices=slices, return_all=True, bc=bc)
    W = lifting(bc) if bc is not None else np.zeros_like(X0, dtype=np.float64)
    todo = range(p) if slices is None else slices
    lam = np.array(dL_dXN, dtype=np.float64, copy=True)
    dg = np.zeros_like(g)
    dalpha = 0.0
    for step in reversed(range(nsteps)):
        Xnext = traj[step + 1]
        lam_prev = np.zeros_like(lam)
        for s in todo:
            ms, bs = sys_[slice_wavenumber(s, p)]
            mu = ms.expand_T(lam[s])
            Lam = bs.solve_T(mu)
            w = ms.rhs_T(Lam)
            lam_prev[s] = w
            if const_g:
                dg[s] += kappa * w
            else:
                dg[step, s] = kappa * w
            Y = np.linalg.lstsq(ms.Sr, np.linalg.lstsq(ms.Sz, (Xnext[s] - W[s]).T, rcond=None)[0].T,
                                rcond=None)[0]
            dS = kappa * (ms.dA @ Y @ ms.B.T + ms.C @ Y @ ms.dD.T)
            if bc is not None:
                dS = dS + kappa * ms.full_apply_dka(W[s])
            dalpha -= float(np.sum(Lam * dS))
        lam = lam_prev
    return lam, dg, dalpha
