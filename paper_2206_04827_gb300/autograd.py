"""torch.autograd wrappers of the heat runs (forward: cyl_heat_step /
cyl_heat_step_bdf, backward: cyl_heat_adjoint / cyl_heat_adjoint_bdf).  torch
supplies device memory and streams only; both passes run in libcyl's CUDA
kernels.

    T_N = heat(T0, g, alpha, dt=..., nsteps=..., ckpt_every=...)
    H_N = heat_bdf(H0, g, alpha, dt, order, nsteps, nvalid=..., ckpt_every=...)

H0 / H_N: [order][p][m][n] histories (slot i = T_{n-i}, slot 0 newest; only
the first nvalid slots of H0 are known, see include/cyl.h: cyl_heat_step_bdf).

T0: [p][m][n] float64 CUDA coefficients (half-complex, see include/cyl.h);
g: one coefficient array (constant forcing) or [nsteps][p][m][n] (g[n] drives
step n -> n+1); alpha: 0-dim float64 tensor; bc: None (zero wall data) or
grid values whose boundary nodes hold time-constant Dirichlet data (no
gradient flows to bc).  Gradients flow to T0, g and alpha.  Plans are
cached per (grid, alpha, dt, tolerance); a new alpha builds a new plan on
the host.
"""
import torch

from . import cyl

_plans = {}


def plan_for(m, n, p, alpha, dt, tol, order=1):
    key = (m, n, p, float(alpha), float(dt), float(tol), int(order), torch.cuda.current_stream().cuda_stream)
    pl = _plans.get(key)
    if pl is None:
        if len(_plans) > 16:
            _plans.clear()
        pl = cyl.Plan(m, n, p, float(alpha), float(dt), tol, poisson=False, heat=True,
                      stream=torch.cuda.current_stream().cuda_stream, bdf_order=int(order))
        _plans[key] = pl
    return pl


class HeatRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, T0, g, alpha, dt, nsteps, ckpt_every, tol, bc):
        p, m, n = T0.shape
        plan = plan_for(m, n, p, alpha.item(), dt, tol)
        T0c = T0.contiguous()
        gc = g.contiguous() if g is not None else None
        stride = 0 if (gc is None or gc.dim() == 3) else p * m * n
        bcc = bc.contiguous() if bc is not None else None
        T = T0c.clone()
        # checkpoints of the forward run, read back by the adjoint (no second forward pass)
        ck = torch.empty((nsteps // ckpt_every + 1) * p * m * n, dtype=torch.float64, device=T0.device)
        plan.heat_step(T, gc, nsteps, g_step_stride=stride, bc=bcc, ckpt=ck, ckpt_every=ckpt_every)
        empty = torch.empty(0, device=T0.device)
        ctx.save_for_backward(T0c, gc if gc is not None else empty, bcc if bcc is not None else empty, ck)
        ctx.meta = (plan, nsteps, ckpt_every, stride, g is not None, bc is not None)
        return T

    @staticmethod
    def backward(ctx, dT):
        T0, gsaved, bcsaved, ck = ctx.saved_tensors
        plan, nsteps, ckpt_every, stride, has_g, has_bc = ctx.meta
        g = gsaved if has_g else None
        dT0 = torch.empty_like(T0)
        dg = torch.empty_like(g) if (has_g and ctx.needs_input_grad[1]) else None
        dal = torch.zeros(1, dtype=torch.float64, device=T0.device) if ctx.needs_input_grad[2] else None
        plan.heat_adjoint(T0, g, nsteps, dT.contiguous(), dT0, dg, dal, g_step_stride=stride,
                          ckpt_every=ckpt_every, bc=bcsaved if has_bc else None, ckpt=ck)
        return (dT0, dg, dal.reshape(()) if dal is not None else None, None, None, None, None, None)


def heat(T0, g, alpha, dt, nsteps, ckpt_every=None, tol=1e-14, bc=None):
    """Differentiable BDF1 run; see the module docstring."""
    if not torch.is_tensor(alpha):
        alpha = torch.tensor(float(alpha), dtype=torch.float64, device=T0.device)
    return HeatRun.apply(T0, g, alpha, float(dt), int(nsteps), int(ckpt_every or nsteps), tol, bc)


class HeatBdfRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H0, g, alpha, dt, order, nsteps, nvalid, ckpt_every, tol, bc):
        _, p, m, n = H0.shape
        plan = plan_for(m, n, p, alpha.item(), dt, tol, order)
        H0c = H0.contiguous()
        gc = g.contiguous() if g is not None else None
        stride = 0 if (gc is None or gc.dim() == 3) else p * m * n
        bcc = bc.contiguous() if bc is not None else None
        H = H0c.clone()
        plan.heat_step_bdf(H, nvalid, gc, nsteps, g_step_stride=stride, bc=bcc)
        empty = torch.empty(0, device=H0.device)
        ctx.save_for_backward(H0c, gc if gc is not None else empty, bcc if bcc is not None else empty)
        ctx.meta = (plan, nsteps, nvalid, ckpt_every, stride, g is not None, bc is not None)
        return H

    @staticmethod
    def backward(ctx, dH):
        H0, gsaved, bcsaved = ctx.saved_tensors
        plan, nsteps, nvalid, ckpt_every, stride, has_g, has_bc = ctx.meta
        g = gsaved if has_g else None
        dH0 = torch.empty_like(H0)
        dg = torch.empty_like(g) if (has_g and ctx.needs_input_grad[1]) else None
        dal = torch.zeros(1, dtype=torch.float64, device=H0.device) if ctx.needs_input_grad[2] else None
        plan.heat_adjoint_bdf(H0, nvalid, g, nsteps, dH.contiguous(), dH0, dg, dal, g_step_stride=stride,
                              ckpt_every=ckpt_every, bc=bcsaved if has_bc else None)
        return (dH0, dg, dal.reshape(()) if dal is not None else None) + (None,) * 7


def heat_bdf(H0, g, alpha, dt, order, nsteps, nvalid=None, ckpt_every=None, tol=1e-14, bc=None):
    """Differentiable BDF run of the given order; see the module docstring."""
    if not torch.is_tensor(alpha):
        alpha = torch.tensor(float(alpha), dtype=torch.float64, device=H0.device)
    return HeatBdfRun.apply(H0, g, alpha, float(dt), int(order), int(nsteps), int(nvalid or order),
                            int(ckpt_every or max(nsteps, 1)), tol, bc)
