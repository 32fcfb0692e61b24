"""Writes large512_sampled.npz: oracle reference values of the 512^3 workload
(one Poisson solve -lap u = f, then 20 BDF1 heat steps with alpha 0.1,
dt 1e-4 and forcing f starting from u) on sampled theta-slices and sampled
coefficients.  Inputs: paper_2206_04827_gb300.inputs.smooth_coeffs(512, 512,
512, decay 1.1) from seed 1002 (the 512^3 workload's generator).  Calls only
oracle/ (QZ Bartels-Stewart with one step of iterative refinement per solve;
the plain direct solve drifts to ~1e-11 at this size; the refinement's
residuals are formed in np.longdouble, whose mantissa width and the machine
are stored with the values).  Slices are independent, so only the sampled
slices are solved.  About 25 minutes on an
8-core host; run from the repository root:

    python tests/golden/make_large512.py
"""
import os
import platform
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import heat  # noqa: E402
from paper_2206_04827_gb300 import inputs  # noqa: E402

P = M = N = 512
ALPHA, DT, HSTEPS, SEED = 0.1, 1e-4, 20, 1002
# wavenumbers 0, 1 (Re), 2 (Im), 127 (Re), 128 (Im), 255 (Re), 256 (Nyquist)
SLICES = [0, 1, 4, 253, 256, 509, 511]
# the large coefficients (low indices) densely, then a few far rows / columns
IDX = sorted(set(range(16)) | {64, 65, 128, 129, 255, 256, 384, 385, 509, 510, 511})


def main():
    f = inputs.smooth_coeffs(P, M, N, 1.1, inputs.rng_for(SEED))
    u = heat.poisson(f, slices=SLICES, refine=1)
    T = heat.heat_steps(u, f, ALPHA, DT, HSTEPS, slices=SLICES, refine=1)
    ix = np.ix_(SLICES, IDX, IDX)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), 'large512_sampled.npz')
    np.savez_compressed(out, slices=np.array(SLICES), idx=np.array(IDX), poisson=u[ix], heat=T[ix],
                        alpha=ALPHA, dt=DT, hsteps=HSTEPS, seed=SEED,
                        longdouble_mantissa_bits=np.finfo(np.longdouble).nmant, machine=platform.machine())
    print('wrote', out)


if __name__ == '__main__':
    main()
