"""Pins of the oracle's Section 3 operators: the printed entries and the
classical identities they encode, evaluated pointwise with scipy.special."""
import os
from fractions import Fraction

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb
from scipy import special

from oracle import operators as ops

GOLDEN = os.path.join(os.path.dirname(__file__), 'golden', 'operators_printed.txt')
BUILD = {'C12': ops.conv_U_to_C2, 'R': ops.mult_r_C2, 'D1': ops.diff1_T_to_U, 'D2': ops.diff2_T_to_C2}


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.split('#')[0].strip()
        if line:
            name, i, j, v = line.split()
            rows.append((name, int(i), int(j), float(Fraction(v))))
    return rows


@pytest.mark.parametrize('name,i,j,v', _golden_rows())
def test_printed_entries(name, i, j, v):
    assert BUILD[name](8)[i, j] == pytest.approx(v, abs=1e-15)


X = np.linspace(-0.97, 0.95, 23)


def _T(c, x):
    return sum(cj * special.eval_chebyt(j, x) for j, cj in enumerate(c))


def _U(c, x):
    return sum(cj * special.eval_chebyu(j, x) for j, cj in enumerate(c))


def _C2(c, x):
    return sum(cj * special.eval_gegenbauer(j, 2.0, x) for j, cj in enumerate(c))


@pytest.mark.parametrize('m', [5, 8, 13])
def test_conversions_pointwise(m):
    rng = np.random.default_rng(m)
    c = rng.standard_normal(m)
    assert np.allclose(_U(ops.conv_T_to_U(m) @ c, X), _T(c, X), atol=1e-12)
    assert np.allclose(_C2(ops.conv_U_to_C2(m) @ c, X), _U(c, X), atol=1e-12)
    assert np.allclose(_C2(ops.conv_T_to_C2(m) @ c, X), _T(c, X), atol=1e-12)


@pytest.mark.parametrize('m', [5, 8, 13])
def test_derivatives_pointwise(m):
    rng = np.random.default_rng(10 + m)
    c = rng.standard_normal(m)
    d1 = npcheb.chebval(X, npcheb.chebder(c, 1))
    d2 = npcheb.chebval(X, npcheb.chebder(c, 2))
    assert np.allclose(_U(ops.diff1_T_to_U(m) @ c, X), d1, atol=1e-10)
    assert np.allclose(_C2(ops.diff2_T_to_C2(m) @ c, X), d2, atol=1e-9)


@pytest.mark.parametrize('m', [6, 9, 14])
def test_multiplication_pointwise(m):
    rng = np.random.default_rng(20 + m)
    c = rng.standard_normal(m)
    c[-2:] = 0.0            # truncated square matrices are exact below the top degree
    assert np.allclose(_C2(ops.mult_r_C2(m) @ c, X), X * _C2(c, X), atol=1e-11)
    assert np.allclose(_C2(ops.r2_C2(m) @ c, X), X ** 2 * _T(c, X), atol=1e-11)


@pytest.mark.parametrize('m,k', [(9, 0), (10, 3), (13, 2)])
def test_radial_operator_pointwise(m, k):
    """R C12 D1 + R^2 D2 - k^2 C02 is r^2 f'' + r f' - k^2 f in the C^(2) basis."""
    rng = np.random.default_rng(30 + m)
    c = rng.standard_normal(m)
    c[-2:] = 0.0
    f = npcheb.chebval(X, c)
    f1 = npcheb.chebval(X, npcheb.chebder(c, 1))
    f2 = npcheb.chebval(X, npcheb.chebder(c, 2))
    want = X ** 2 * f2 + X * f1 - k ** 2 * f
    assert np.allclose(_C2(ops.radial_laplacian_r2(m, k) @ c, X), want, atol=1e-9)


def test_dirichlet_basis_vanishes_at_ends():
    S = ops.dirichlet_basis(11)
    for j in range(9):
        assert _T(S[:, j], np.array([-1.0, 1.0])) == pytest.approx([0.0, 0.0], abs=1e-14)
    assert np.linalg.matrix_rank(S) == 9


def test_printed_C01_is_not_the_conversion():
    """The printed C01 (zero diagonal, 1/2 off-diagonal) fails the T -> U
    identity the text states for it; the oracle's conversion passes it.  This
    pins the reading of the garbled matrix."""
    m = 7
    printed = 0.5 * (np.eye(m, k=1) + np.eye(m, k=-1))
    rng = np.random.default_rng(3)
    c = rng.standard_normal(m)
    assert not np.allclose(_U(printed @ c, X), _T(c, X), atol=1e-6)
    assert np.allclose(_U(ops.conv_T_to_U(m) @ c, X), _T(c, X), atol=1e-12)
