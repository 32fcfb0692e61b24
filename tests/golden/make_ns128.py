"""Writes ns128_sampled.npz: reference values of one Navier-Stokes step of the
128^3 workload (Section 4, IMEX BDF1 in poloidal-toroidal form; Re 100,
dt 1e-3) from the workload's seeded potentials (inputs.smooth_coeffs(128,
128, 128, decay 1.25), seed 1005, lambda_w then gamma_w), on sampled
theta-slices and coefficients.  Calls only oracle/: the reference is the
extended-precision step (oracle.ns, extended=True: the nonlinear term in
np.longdouble, refined solves), and the file also stores how far the plain
FP64 oracle step lands from it over the whole field -- the rounding floor of
an FP64 evaluation of these formulas, which the GPU check is measured
against.  The long-double mantissa width and the machine are stored with the
values.  About five minutes on an 8-core host; run from the repository root:

    python tests/golden/make_ns128.py
"""
import os
import platform
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ns  # noqa: E402
from paper_2206_04827_gb300 import inputs  # noqa: E402

L, RE, DT, SEED = 128, 100.0, 1e-3, 1005
# wavenumbers 0, 1, 2, 3 (Re and Im), 32, 63, Nyquist
SLICES = [0, 1, 2, 3, 4, 5, 6, 63, 64, 125, 126, 127]
IDX = sorted(set(range(16)) | {31, 32, 47, 48, 63, 64, 95, 96, 111, 126, 127})


def main():
    if np.finfo(np.longdouble).nmant < 63:
        raise SystemExit('np.longdouble is not wider than double on this machine')
    rng = inputs.rng_for(SEED)
    Lw = inputs.smooth_coeffs(L, L, L, 1.25, rng)
    Gw = inputs.smooth_coeffs(L, L, L, 1.25, rng)
    ref_l, ref_g = ns.ns_steps(Lw, Gw, RE, DT, 1, extended=True)
    f64_l, f64_g = ns.ns_steps(Lw, Gw, RE, DT, 1)
    rel = lambda a, b: float(np.abs(a - b).max() / np.abs(b).max())
    ix = np.ix_(SLICES, IDX, IDX)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), 'ns128_sampled.npz')
    np.savez_compressed(out, slices=np.array(SLICES), idx=np.array(IDX), lam=ref_l[ix], gam=ref_g[ix],
                        lam_max=np.abs(ref_l).max(), gam_max=np.abs(ref_g).max(),
                        fp64_err_lam=rel(f64_l, ref_l), fp64_err_gam=rel(f64_g, ref_g),
                        fp64_err_lam_sampled=float(np.abs(f64_l[ix] - ref_l[ix]).max() / np.abs(ref_l).max()),
                        fp64_err_gam_sampled=float(np.abs(f64_g[ix] - ref_g[ix]).max() / np.abs(ref_g).max()),
                        Re=RE, dt=DT, seed=SEED, decay=1.25,
                        longdouble_mantissa_bits=np.finfo(np.longdouble).nmant, machine=platform.machine())
    print('wrote', out, 'FP64 oracle vs reference: lambda %.2e, gamma %.2e' % (rel(f64_l, ref_l), rel(f64_g, ref_g)))


if __name__ == '__main__':
    main()
