"""Writes heat256_sampled.npz: oracle reference values of a 256^3 BDF1 run
(alpha 0.2, dt 1e-4, 5 steps, T0 and g = smooth coefficients with decay
1.15 from seed 77, in that draw order) on sampled theta-slices and sampled
coefficients.  Calls only oracle/ (QZ Bartels-Stewart with two steps of
iterative refinement per solve, residuals in extended precision: at this
size the plain direct solve drifts by ~3e-12 over the 5 steps on the k = 0
slice).  The platform's extended precision (mantissa bits of np.longdouble)
is stored with the values.  About a minute; run from the repository root:

    python tests/golden/make_heat256.py
"""
import os
import platform
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import heat  # noqa: E402
from paper_2206_04827_gb300 import inputs  # noqa: E402

P = M = N = 256
ALPHA, DT, STEPS, SEED, DECAY = 0.2, 1e-4, 5, 77, 1.15
SLICES = [0, 1, 2, 127, 254, 255]
IDX = sorted(set(range(16)) | {64, 65, 127, 128, 191, 192, 253, 254, 255})


def main():
    rng = inputs.rng_for(SEED)
    X0 = inputs.smooth_coeffs(P, M, N, DECAY, rng)
    g = inputs.smooth_coeffs(P, M, N, DECAY, rng)
    T = heat.heat_steps(X0, g, ALPHA, DT, STEPS, slices=SLICES, refine=2)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), 'heat256_sampled.npz')
    np.savez_compressed(out, slices=np.array(SLICES), idx=np.array(IDX), heat=T[np.ix_(SLICES, IDX, IDX)],
                        alpha=ALPHA, dt=DT, steps=STEPS, seed=SEED, decay=DECAY,
                        longdouble_mantissa_bits=np.finfo(np.longdouble).nmant, machine=platform.machine())
    print('wrote', out)


if __name__ == '__main__':
    main()
