"""Doubled CCF grid (oracle; test infrastructure only).

Section 2, Definition "grid": x_(j,k,l) = (cos((m-j-1)pi/(m-1)),
cos((n-k-1)pi/(n-1)), (2l-p)pi/p), 0 <= j < m, 0 <= k < n, 0 <= l < p.
Section 2, CCF polynomial: the Fourier factor of basis index l is
exp(i (l - floor(p/2)) theta).
"""
import numpy as np


def cheb_points(m):
    """Radial (or vertical) grid of Definition "grid": ascending on [-1, 1]."""
    j = np.arange(m, dtype=np.float64)
    return np.cos((m - j - 1.0) * np.pi / (m - 1.0))


def theta_points(p):
    """Angular grid of Definition "grid": theta_l = (2l - p) pi / p."""
    l = np.arange(p, dtype=np.float64)
    return (2.0 * l - p) * np.pi / p


def wavenumbers(p):
    """Wavenumber k = l - floor(p/2) carried by basis index l (Section 2)."""
    return np.arange(p) - p // 2
