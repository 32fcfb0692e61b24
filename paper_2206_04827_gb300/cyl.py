"""ctypes binding of libcyl (argument marshalling only: every step of the
solver runs in the library's CUDA kernels).

Importing this module loads ``libcyl.so`` from the package directory and
raises ImportError when it has not been built (``python -m
paper_2206_04827_gb300.build``); there is no fallback implementation.

Device arrays are passed as torch CUDA tensors (float64, contiguous, layout
[p][m][n]); torch supplies the memory and the stream, nothing else.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, 'libcyl.so')

if not os.path.exists(LIB_PATH):
    raise ImportError('libcyl.so is not built (run python -m paper_2206_04827_gb300.build)')
_lib = ctypes.CDLL(LIB_PATH)

# status codes and flags (include/cyl.h)
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ESTATE = range(6)
WITH_POISSON, WITH_HEAT, BOTH_PARITIES, HOST_ONLY, FORCE_GLOBAL, TEST_NO_TMA, WITH_BC = 1, 2, 4, 8, 16, 32, 64
PLAIN_SWEEPS, WITH_DISK, FORCE_CLUSTER = 128, 256, 512
VALUES, COEFFS = 0, 1

_c_double_p = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p
_sig = {
    'cyl_plan': (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_uint, _vp]),
    'cyl_plan_bdf': (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_uint, _vp]),
    'cyl_heat_step_bdf': (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, ctypes.c_longlong, ctypes.c_int, _vp]),
    'cyl_heat_adjoint_bdf': (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, ctypes.c_longlong, ctypes.c_int, _vp,
                                            ctypes.c_int, _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t]),
    'cyl_heat_adjoint_bdf_workspace': (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                      ctypes.POINTER(ctypes.c_size_t)]),
    'cyl_plan_launch_info': (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    'cyl_plan_item_tables': (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int), _c_double_p, _c_double_p]),
    'cyl_disk_poisson': (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int]),
    'cyl_destroy': (ctypes.c_int, [_vp]),
    'cyl_vals2coeffs': (ctypes.c_int, [_vp, _vp, _vp]),
    'cyl_coeffs2vals': (ctypes.c_int, [_vp, _vp, _vp]),
    'cyl_poisson': (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int]),
    'cyl_heat_step': (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_longlong, ctypes.c_int, _vp, ctypes.c_int]),
    'cyl_heat_step_bc': (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_longlong, ctypes.c_int, _vp, _vp, ctypes.c_int]),
    'cyl_heat_adjoint': (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _vp, _vp,
                                        _vp, _vp, _vp, ctypes.c_size_t]),
    'cyl_heat_adjoint_bc': (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_longlong, ctypes.c_int, _vp, ctypes.c_int, _vp,
                                           _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t]),
    'cyl_heat_adjoint_workspace': (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                  ctypes.POINTER(ctypes.c_size_t)]),
    'cyl_status_string': (ctypes.c_char_p, [ctypes.c_int]),
    'cyl_sync': (ctypes.c_int, [_vp]),
    'cyl_plan_shifts': (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       _c_double_p, _c_double_p, _c_double_p]),
    'cyl_plan_operator': (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int), _c_double_p]),
    'cyl_grid': (ctypes.c_int, [_vp, _c_double_p, _c_double_p, _c_double_p]),
    'cyl_plan_flops': (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _c_double_p]),
    'cyl_plan_batch': (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.c_double,
                                      ctypes.c_uint, _vp]),
    'cyl_batch_layout': (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong)]),
    'cyl_heat_step_batch': (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int]),
    'cyl_batch_set_config': (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    'cyl_batch_get_config': (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    'cyl_batch_autotune': (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    'cyl_ellip_K': (ctypes.c_double, [ctypes.c_double]),
    'cyl_jacobi_dn': (ctypes.c_double, [ctypes.c_double, ctypes.c_double]),
    'cyl_ns_workspace': (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    'cyl_ns_step': (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp, ctypes.c_size_t]),
    'cyl_xform_table': (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _c_double_p]),
    'cyl_fp64_fma_probe': (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_longlong, _vp, _c_double_p, _vp]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class CylError(RuntimeError):
    def __init__(self, status, what):
        super().__init__('%s: %s' % (what, _lib.cyl_status_string(status).decode()))
        self.status = status


def _check(status, what):
    if status != OK:
        raise CylError(status, what)


def status_string(s):
    return _lib.cyl_status_string(s).decode()


def ellip_K(kprime):
    return _lib.cyl_ellip_K(kprime)


def jacobi_dn(u, kprime):
    return _lib.cyl_jacobi_dn(u, kprime)


def _ptr(t, name, numel=None):
    """Device pointer of a contiguous float64 CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not (t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()):
        raise ValueError('%s must be a contiguous float64 CUDA tensor' % name)
    if numel is not None and t.numel() < numel:
        raise ValueError('%s holds %d elements, needs %d' % (name, t.numel(), numel))
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """Owner of one ``cyl_plan_t`` (see include/cyl.h: cyl_plan)."""

    def __init__(self, n_r, n_z, n_theta, alpha=0.0, dt=0.0, adi_tol=1e-14, poisson=True, heat=False,
                 both_parities=False, host_only=False, force_global=False, stream=None, extra_flags=0,
                 bdf_order=1):
        flags = (WITH_POISSON if poisson else 0) | (WITH_HEAT if heat else 0) \
            | (BOTH_PARITIES if both_parities else 0) | (HOST_ONLY if host_only else 0) \
            | (FORCE_GLOBAL if force_global else 0) | int(extra_flags)
        if stream is None and not host_only:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self._h = _vp()
        _check(_lib.cyl_plan_bdf(ctypes.byref(self._h), int(n_r), int(n_z), int(n_theta), float(alpha), float(dt),
                                 float(adi_tol), int(bdf_order), flags, _vp(stream) if stream else None),
               'cyl_plan_bdf')
        self.m, self.n, self.p = int(n_r), int(n_z), int(n_theta)
        self.bdf_order = int(bdf_order)
        self.N = self.m * self.n * self.p
        self.alpha, self.dt = float(alpha), float(dt)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _lib.cyl_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- device calls -------------------------------------------------------
    def vals2coeffs(self, vals, coeffs):
        _check(_lib.cyl_vals2coeffs(self._h, _ptr(vals, 'vals', self.N), _ptr(coeffs, 'coeffs', self.N)),
               'cyl_vals2coeffs')
        return coeffs

    def coeffs2vals(self, coeffs, vals):
        _check(_lib.cyl_coeffs2vals(self._h, _ptr(coeffs, 'coeffs', self.N), _ptr(vals, 'vals', self.N)),
               'cyl_coeffs2vals')
        return vals

    def poisson(self, f, u, space=COEFFS, bc=None):
        """-lap u = f; bc: None (zero wall data) or grid values whose boundary
        nodes hold the Dirichlet data (include/cyl.h: cyl_poisson)."""
        _check(_lib.cyl_poisson(self._h, _ptr(f, 'f', self.N), _ptr(bc, 'bc', self.N), _ptr(u, 'u', self.N),
                                int(space)), 'cyl_poisson')
        return u

    def disk_poisson(self, f, u, space=COEFFS):
        """-Delta_h u = f, the horizontal (disk) Poisson solve (include/cyl.h: cyl_disk_poisson)."""
        _check(_lib.cyl_disk_poisson(self._h, _ptr(f, 'f', self.N), _ptr(u, 'u', self.N), int(space)),
               'cyl_disk_poisson')
        return u

    def heat_step(self, T, g=None, nsteps=1, g_step_stride=0, ckpt=None, ckpt_every=1, bc=None):
        need = None if ckpt is None else (nsteps // ckpt_every + 1) * self.N
        _check(_lib.cyl_heat_step_bc(self._h, _ptr(T, 'T', self.N), _ptr(g, 'g', self.N), int(g_step_stride),
                                     int(nsteps), _ptr(bc, 'bc', self.N), _ptr(ckpt, 'ckpt', need),
                                     int(ckpt_every)), 'cyl_heat_step_bc')
        return T

    def heat_step_bdf(self, hist, nvalid, g=None, nsteps=1, g_step_stride=0, bc=None):
        """nsteps steps of the plan's BDF order on the history hist (bdf_order x N
        coefficients, slot 0 = newest; include/cyl.h: cyl_heat_step_bdf)."""
        _check(_lib.cyl_heat_step_bdf(self._h, _ptr(hist, 'hist', self.bdf_order * self.N), int(nvalid),
                                      _ptr(g, 'g', self.N), int(g_step_stride), int(nsteps),
                                      _ptr(bc, 'bc', self.N)), 'cyl_heat_step_bdf')
        return hist

    def heat_adjoint_bdf(self, hist0, nvalid, g, nsteps, dL_dhistN, dL_dhist0, dL_dg=None, dL_dalpha=None,
                         g_step_stride=0, ckpt_every=1, bc=None, workspace=None):
        """Reverse-mode gradients of a BDF run (include/cyl.h: cyl_heat_adjoint_bdf).
        The workspace tensor is allocated here (torch) when not given."""
        nb = ctypes.c_size_t()
        _check(_lib.cyl_heat_adjoint_bdf_workspace(self._h, int(nsteps), int(ckpt_every), int(dL_dalpha is not None),
                                                   ctypes.byref(nb)), 'cyl_heat_adjoint_bdf_workspace')
        nbytes = nb.value
        if workspace is None:
            import torch
            workspace = torch.empty((nbytes + 7) // 8, dtype=torch.float64, device=dL_dhist0.device)
        bN = self.bdf_order * self.N
        _check(_lib.cyl_heat_adjoint_bdf(self._h, _ptr(hist0, 'hist0', bN), int(nvalid), _ptr(g, 'g', self.N),
                                         int(g_step_stride), int(nsteps), _ptr(bc, 'bc', self.N), int(ckpt_every),
                                         _ptr(dL_dhistN, 'dL_dhistN', bN), _ptr(dL_dhist0, 'dL_dhist0', bN),
                                         _ptr(dL_dg, 'dL_dg', self.N), _ptr(dL_dalpha, 'dL_dalpha', 1),
                                         _ptr(workspace, 'workspace', (nbytes + 7) // 8), ctypes.c_size_t(nbytes)),
               'cyl_heat_adjoint_bdf')
        return dL_dhist0

    def adjoint_workspace_bytes(self, nsteps, ckpt_every, need_alpha, have_ckpt=False):
        mode = 0 if not need_alpha else (2 if have_ckpt else 1)
        nb = ctypes.c_size_t()
        _check(_lib.cyl_heat_adjoint_workspace(self._h, int(nsteps), int(ckpt_every), mode, ctypes.byref(nb)),
               'cyl_heat_adjoint_workspace')
        return nb.value

    def heat_adjoint(self, T0, g, nsteps, dL_dTN, dL_dT0, dL_dg=None, dL_dalpha=None, g_step_stride=0,
                     ckpt_every=1, workspace=None, bc=None, ckpt=None):
        """Reverse-mode gradients of the BDF1 run (see include/cyl.h: cyl_heat_adjoint, _bc).
        ckpt: the checkpoints the forward run wrote with the same ckpt_every (saves
        the adjoint's own checkpoint pass).  The workspace tensor is allocated here
        (torch) when not given."""
        nbytes = self.adjoint_workspace_bytes(nsteps, ckpt_every, dL_dalpha is not None, ckpt is not None)
        nck = (int(nsteps) // int(ckpt_every) + 1) * self.N
        if nbytes and workspace is None:
            import torch
            workspace = torch.empty((nbytes + 7) // 8, dtype=torch.float64, device=dL_dT0.device)
        _check(_lib.cyl_heat_adjoint_bc(self._h, _ptr(T0, 'T0', self.N), _ptr(g, 'g', self.N), int(g_step_stride),
                                     int(nsteps), _ptr(bc, 'bc', self.N), int(ckpt_every), _ptr(ckpt, 'ckpt', nck),
                                     _ptr(dL_dTN, 'dL_dTN', self.N),
                                     _ptr(dL_dT0, 'dL_dT0', self.N), _ptr(dL_dg, 'dL_dg', self.N),
                                     _ptr(dL_dalpha, 'dL_dalpha', 1),
                                     _ptr(workspace, 'workspace', (nbytes + 7) // 8) if nbytes else None,
                                     ctypes.c_size_t(nbytes)), 'cyl_heat_adjoint_bc')
        return dL_dT0

    def ns_workspace_bytes(self):
        nb = ctypes.c_size_t()
        _check(_lib.cyl_ns_workspace(self._h, ctypes.byref(nb)), 'cyl_ns_workspace')
        return nb.value

    def ns_step(self, lam_w, gam_w, nsteps=1, workspace=None):
        """nsteps Navier-Stokes steps on the vorticity PT state (include/cyl.h:
        cyl_ns_step); the plan needs poisson, heat and disk tables, alpha = 1/Re.
        The workspace tensor is allocated here (torch) when not given."""
        nbytes = self.ns_workspace_bytes()
        if workspace is None:
            import torch
            workspace = torch.empty((nbytes + 7) // 8, dtype=torch.float64, device=lam_w.device)
        _check(_lib.cyl_ns_step(self._h, _ptr(lam_w, 'lam_w', self.N), _ptr(gam_w, 'gam_w', self.N), int(nsteps),
                                _ptr(workspace, 'workspace', (nbytes + 7) // 8), ctypes.c_size_t(nbytes)),
               'cyl_ns_step')
        return lam_w, gam_w

    def sync(self):
        """Wait for the plan's stream; raise on a device-side timeout or CUDA error."""
        _check(_lib.cyl_sync(self._h), 'cyl_sync')

    # -- host introspection ---------------------------------------------------
    def grid(self):
        """(r, z, theta) of the doubled grid (host arrays)."""
        r = (ctypes.c_double * self.m)()
        z = (ctypes.c_double * self.n)()
        t = (ctypes.c_double * self.p)()
        _check(_lib.cyl_grid(self._h, r, z, t), 'cyl_grid')
        return np.array(r), np.array(z), np.array(t)

    def flops(self, which, nsteps, transposed=False):
        """Algorithmic FP64 flops of nsteps steps (see include/cyl.h: cyl_plan_flops)."""
        return plan_flops(self._h, which, nsteps, transposed)

    def shifts(self, which, k, parity):
        """(J, (a, b, c, d), p_shifts, q_shifts) of one wavenumber (host tables)."""
        J = ctypes.c_int()
        _check(_lib.cyl_plan_shifts(self._h, which, k, parity, ctypes.byref(J), None, None, None), 'cyl_plan_shifts')
        iv = (ctypes.c_double * 4)()
        ps = (ctypes.c_double * J.value)()
        qs = (ctypes.c_double * J.value)()
        _check(_lib.cyl_plan_shifts(self._h, which, k, parity, ctypes.byref(J), iv, ps, qs), 'cyl_plan_shifts')
        return J.value, tuple(iv), np.array(ps), np.array(qs)

    def launch_info(self, which):
        """Launch layout of one kind's ADI kernel (see include/cyl.h: cyl_plan_launch_info)."""
        info = (ctypes.c_int * 9)()
        _check(_lib.cyl_plan_launch_info(self._h, which, info), 'cyl_plan_launch_info')
        keys = ('items', 'threads', 'twist_half', 'placement', 'smem', 'ctas_per_item', 'slices', 'built',
                'all_twisted')
        return dict(zip(keys, list(info)))

    def item_tables(self, which, item, j, transposed=False):
        """(info dict, radial records, vertical records) of one item's ADI iteration j
        (of the transposed system of the adjoint when transposed)."""
        info = (ctypes.c_int * 8)()
        tr = int(bool(transposed))
        _check(_lib.cyl_plan_item_tables(self._h, which, item, j, tr, info, None, None), 'cyl_plan_item_tables')
        M, Nz, J, twr, twz = info[0], info[1], info[2], info[3], info[4]
        rad = (ctypes.c_double * (M * 12 + (24 if twr else 0)))()
        ver = (ctypes.c_double * (Nz * 8 + (16 if twz else 0)))()
        _check(_lib.cyl_plan_item_tables(self._h, which, item, j, tr, info, rad, ver), 'cyl_plan_item_tables')
        keys = ('M', 'Nz', 'J', 'twr', 'twz', 'k', 'pr', 'pz')
        return dict(zip(keys, list(info))), np.array(rad), np.array(ver)

    def operator(self, op, which, k, parity):
        """Dense parity block of A (op 0), C (1), B (2) or D (3)."""
        d = ctypes.c_int()
        _check(_lib.cyl_plan_operator(self._h, op, which, k, parity, ctypes.byref(d), None), 'cyl_plan_operator')
        buf = (ctypes.c_double * (d.value * d.value))()
        _check(_lib.cyl_plan_operator(self._h, op, which, k, parity, ctypes.byref(d), buf), 'cyl_plan_operator')
        return np.array(buf).reshape(d.value, d.value)


class BatchPlan:
    """Owner of a batch plan (see include/cyl.h: cyl_plan_batch)."""

    def __init__(self, n_r, n_z, n_theta, alpha, dt, adi_tol=1e-14, both_parities=False, stream=None,
                 plain_sweeps=False, host_only=False):
        k = len(n_r)
        if stream is None and not host_only:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        ia = lambda v: (ctypes.c_int * k)(*[int(x) for x in v])
        self._h = _vp()
        _check(_lib.cyl_plan_batch(ctypes.byref(self._h), k, ia(n_r), ia(n_z), ia(n_theta),
                                   (ctypes.c_double * k)(*[float(a) for a in alpha]), float(dt), float(adi_tol),
                                   WITH_HEAT | (BOTH_PARITIES if both_parities else 0)
                                   | (PLAIN_SWEEPS if plain_sweeps else 0) | (HOST_ONLY if host_only else 0),
                                   _vp(stream) if stream else None),
               'cyl_plan_batch')
        offs = (ctypes.c_longlong * (k + 1))()
        _check(_lib.cyl_batch_layout(self._h, None, offs), 'cyl_batch_layout')
        self.offsets = [int(o) for o in offs]
        self.shapes = [(int(p), int(m), int(n)) for m, n, p in zip(n_r, n_z, n_theta)]
        self.N = self.offsets[-1]

    def close(self):
        if self._h:
            _lib.cyl_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def heat_step(self, T, g=None, nsteps=1):
        _check(_lib.cyl_heat_step_batch(self._h, _ptr(T, 'T', self.N), _ptr(g, 'g', self.N), int(nsteps)),
               'cyl_heat_step_batch')
        return T

    def set_config(self, threshold, groups, chains_per_thread=1):
        _check(_lib.cyl_batch_set_config(self._h, int(threshold), int(groups), int(chains_per_thread)),
               'cyl_batch_set_config')

    def config(self):
        """(threshold, groups, items per class); chains_per_thread() gives the third knob."""
        t, g, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ipc = (ctypes.c_int * 2)()
        _check(_lib.cyl_batch_get_config(self._h, ctypes.byref(t), ctypes.byref(g), ctypes.byref(c), ipc),
               'cyl_batch_get_config')
        self._cpt = c.value
        return t.value, g.value, (ipc[0], ipc[1])

    def chains_per_thread(self):
        self.config()
        return self._cpt

    def autotune(self, T, g=None, nsteps=1):
        ms = ctypes.c_double()
        _check(_lib.cyl_batch_autotune(self._h, _ptr(T, 'T', self.N), _ptr(g, 'g', self.N), int(nsteps),
                                       ctypes.byref(ms)), 'cyl_batch_autotune')
        return ms.value

    def sync(self):
        _check(_lib.cyl_sync(self._h), 'cyl_sync')

    def flops(self, nsteps):
        return plan_flops(self._h, 1, nsteps, False)

    def view(self, T, i):
        """Problem i's [p][m][n] view of a batch array."""
        p, m, n = self.shapes[i]
        return T[self.offsets[i]:self.offsets[i + 1]].view(p, m, n)


def plan_flops(handle, which, nsteps, transposed):
    f = ctypes.c_double()
    _check(_lib.cyl_plan_flops(handle, int(which), int(nsteps), int(bool(transposed)), ctypes.byref(f)),
           'cyl_plan_flops')
    return f.value


def xform_table(kind, L):
    """(info dict, table) of one chirp-z line transform (include/cyl.h: cyl_xform_table)."""
    info = (ctypes.c_int * 11)()
    _check(_lib.cyl_xform_table(int(kind), int(L), info, None), 'cyl_xform_table')
    tab = (ctypes.c_double * info[10])()
    _check(_lib.cyl_xform_table(int(kind), int(L), info, tab), 'cyl_xform_table')
    keys = ('P', 'logP', 'A', 'B', 'ia0', 'jb0', 'pre_off', 'post_off', 'H_off', 'tw_off', 'size')
    return dict(zip(keys, list(info))), np.array(tab)


def fp64_fma_probe(sink, blocks, threads, iters, stream):
    """Launch the FP64 FMA-throughput probe (include/cyl.h: cyl_fp64_fma_probe) on
    `stream`; returns the launch's FP64 flops.  The caller times it."""
    f = ctypes.c_double()
    _check(_lib.cyl_fp64_fma_probe(int(blocks), int(threads), int(iters), _ptr(sink, 'sink', blocks * threads),
                                   ctypes.byref(f), _vp(stream)), 'cyl_fp64_fma_probe')
    return f.value


def exported_symbols():
    """Names of the functions the binding requires from libcyl."""
    return sorted(_sig)
