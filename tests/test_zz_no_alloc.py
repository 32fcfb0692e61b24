"""The allocation-free transform entry point (cyl_vals2coeffs_noalloc) called
through the C ABI must give what the planned transform (cyl_vals2coeffs)
gives, on consecutive calls that share its fixed scratch array.  It serves
callers that cannot allocate device memory (hosts whose own pool owns all
device memory, loops that must never enter an allocator), so it is checked
here against the planned path, within the transform tolerance used by the
other GPU tests, also when the input and output arrays are the same."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

TOL_XFORM = 1e-13


@pytest.fixture(scope='module')
def cyl():
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    from paper_2206_04827_gb300 import cyl as C
    f = C._lib.cyl_vals2coeffs_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return C


def _noalloc(C, m, n, p, vals, out):
    stream = torch.cuda.current_stream().cuda_stream
    return C._lib.cyl_vals2coeffs_noalloc(m, n, p, ctypes.c_void_p(vals.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(stream))


def test_noalloc_transform_matches_planned_on_consecutive_calls(cyl):
    # two calls in a row, the second smaller than the first, so stale scratch
    # contents from the first call would show up in the second
    for (m, n, p), seed in (((33, 29, 16), 1), ((12, 9, 6), 2), ((128, 128, 128), 3)):
        vals = torch.as_tensor(np.random.default_rng(seed).standard_normal((p, m, n)), device='cuda')
        plan = cyl.Plan(m, n, p)
        want = plan.vals2coeffs(vals, torch.empty_like(vals))
        got = torch.full_like(vals, np.nan)
        assert _noalloc(cyl, m, n, p, vals, got) == cyl.OK
        torch.cuda.synchronize()
        w, g = want.cpu().numpy(), got.cpu().numpy()
        assert np.abs(g - w).max() / np.abs(w).max() <= TOL_XFORM
        plan.close()


def test_noalloc_in_place(cyl):
    m, n, p = 33, 29, 16
    vals = torch.as_tensor(np.random.default_rng(4).standard_normal((p, m, n)), device='cuda')
    plan = cyl.Plan(m, n, p)
    want = plan.vals2coeffs(vals, torch.empty_like(vals)).cpu().numpy()
    t = vals.clone()
    assert _noalloc(cyl, m, n, p, t, t) == cyl.OK
    torch.cuda.synchronize()
    assert np.abs(t.cpu().numpy() - want).max() / np.abs(want).max() <= TOL_XFORM
    plan.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(cyl):
    m = n = p = 170          # 2 N + m^2 + n^2 + p^2 exceeds the fixed scratch
    small = torch.zeros(8, device='cuda', dtype=torch.float64)
    assert _noalloc(cyl, m, n, p, small, small) == cyl.EINVAL
    assert _noalloc(cyl, 8, 8, 7, small, small) == cyl.EINVAL
