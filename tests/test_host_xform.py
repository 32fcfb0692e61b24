"""Host logic of the chirp-z value <-> coefficient transforms (Section 2: the
DCT-I in r and z, the DFT in theta), on the CPU: the library's own table
blocks (cyl_xform_table) driven through an emulation of the transform
kernel's dataflow -- inputs times the pre-multipliers at their circular
slots, a radix-2 decimation-in-frequency FFT with the table's twiddles
(natural order in, bit-reversed out), the product with the bit-reversed
kernel spectrum, a decimation-in-time inverse FFT with conjugate twiddles,
the post-multipliers, the real part (DCT-I) or the separation of two lines
packed in one complex FFT (DFT) -- three passes (z, r, theta) compared with
the oracle's direct-sum transforms."""
import os

import numpy as np
import pytest

from oracle import transforms as otr


@pytest.fixture(scope='module')
def cyl():
    from paper_2206_04827_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    from paper_2206_04827_gb300 import cyl as C
    return C


def _cplx(tab, off, count):
    return tab[off:off + 2 * count].reshape(count, 2) @ np.array([1.0, 1j])


def _dif(buf, tw, logP):
    P = buf.shape[1]
    for lh in reversed(range(logP)):
        h = 1 << lh
        w = tw[np.arange(h) * ((P // 2) >> lh)]
        v = buf.reshape(buf.shape[0], P // (2 * h), 2, h)
        x0, x1 = v[:, :, 0, :].copy(), v[:, :, 1, :].copy()
        v[:, :, 0, :] = x0 + x1
        v[:, :, 1, :] = (x0 - x1) * w
    return buf


def _dit_inv(buf, tw, logP):
    P = buf.shape[1]
    for lh in range(logP):
        h = 1 << lh
        w = np.conj(tw[np.arange(h) * ((P // 2) >> lh)])
        v = buf.reshape(buf.shape[0], P // (2 * h), 2, h)
        x0, t = v[:, :, 0, :].copy(), v[:, :, 1, :] * w
        v[:, :, 0, :] = x0 + t
        v[:, :, 1, :] = x0 - t
    return buf


def _emulate(cyl, kind, lines):
    """One pass of the kernel over real lines [nl][L]."""
    info, tab = cyl.xform_table(kind, lines.shape[1])
    P, logP, A, B, ia0, jb0 = (info[k] for k in ('P', 'logP', 'A', 'B', 'ia0', 'jb0'))
    pre = _cplx(tab, info['pre_off'], A)
    post = _cplx(tab, info['post_off'], B)
    Hbr = _cplx(tab, info['H_off'], P)
    tw = _cplx(tab, info['tw_off'], P // 2)
    L = lines.shape[1]
    nl = lines.shape[0]
    if kind <= 1:
        x = lines.astype(complex)
    else:
        pad = np.vstack([lines, np.zeros((nl % 2, L))])
        a, b = pad[0::2], pad[1::2]
        if kind == 2:
            x = a + 1j * b
        else:
            def herm(hc):             # half-complex slots -> C_w, w = -L/2 .. L/2-1
                C = np.zeros((hc.shape[0], L), dtype=complex)
                for idx, w in enumerate(range(-L // 2, L // 2)):
                    v = abs(w)
                    if v == 0:
                        C[:, idx] = hc[:, 0]
                    elif v == L // 2:
                        C[:, idx] = hc[:, L - 1]
                    else:
                        c = hc[:, 2 * v - 1] + 1j * hc[:, 2 * v]
                        C[:, idx] = c if w > 0 else np.conj(c)
                return C
            x = herm(a) + 1j * herm(b)
    buf = np.zeros((x.shape[0], P), dtype=complex)
    buf[:, (ia0 + np.arange(A)) % P] = pre * x
    buf = _dit_inv(_dif(buf, tw, logP) * Hbr, tw, logP)
    Z = post * buf[:, (jb0 + np.arange(B)) % P]
    if kind <= 1:
        return Z.real
    if kind == 3:
        out = np.empty((2 * Z.shape[0], L))
        out[0::2], out[1::2] = Z.real, Z.imag
        return out[:nl]
    out = np.empty((2 * Z.shape[0], L))
    for s in range(L):
        w = 0 if s == 0 else (L // 2 if s == L - 1 else (s + 1) // 2)
        Zw = Z[:, w - jb0]
        if w in (0, L // 2):
            f, g = Zw.real, Zw.imag
        else:
            Zm = Z[:, -w - jb0]
            F = 0.5 * (Zw + np.conj(Zm))
            G = (Zw - np.conj(Zm)) / 2j
            f, g = (F.imag, G.imag) if s % 2 == 0 else (F.real, G.real)
        out[0::2, s], out[1::2, s] = f, g
    return out[:nl]


def _pass(cyl, kind, X, axis):
    Y = np.moveaxis(X, axis, -1)
    shp = Y.shape
    out = _emulate(cyl, kind, Y.reshape(-1, shp[-1]))
    return np.moveaxis(out.reshape(shp), -1, axis)


@pytest.mark.parametrize("p,m,n", [(2, 4, 5), (6, 5, 9), (8, 17, 12), (16, 33, 40), (10, 128, 7), (4, 9, 512), (512, 5, 4), (30, 6, 7)])
def test_emulated_chirp_transforms_match_oracle(cyl, p, m, n):
    rng = np.random.default_rng(p * 1000 + m * 10 + n)
    vals = rng.standard_normal((p, m, n))
    c = _pass(cyl, 2, _pass(cyl, 0, _pass(cyl, 0, vals, 2), 1), 0)
    want = otr.vals2coeffs(vals)
    assert np.abs(c - want).max() / np.abs(want).max() <= 1e-13
    H = rng.standard_normal((p, m, n))
    v = _pass(cyl, 1, _pass(cyl, 1, _pass(cyl, 3, H, 0), 1), 2)
    want = otr.coeffs2vals(H)
    assert np.abs(v - want).max() / np.abs(want).max() <= 1e-13


def test_xform_table_sizes_and_arguments(cyl):
    info, _ = cyl.xform_table(0, 128)
    assert info['P'] == 256 and info['A'] == info['B'] == 128       # P >= 2L - 1
    info, _ = cyl.xform_table(2, 128)
    assert info['P'] == 256 and info['jb0'] == -63                  # outputs w = -63 .. 64
    info, _ = cyl.xform_table(3, 512)
    assert info['P'] == 1024 and info['ia0'] == -256
    for bad in ((0, 1), (2, 7), (4, 8), (0, 5000)):
        with pytest.raises(cyl.CylError):
            cyl.xform_table(*bad)
