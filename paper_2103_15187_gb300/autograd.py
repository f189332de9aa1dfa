"""torch.autograd wrapper of a multi-step window of the fractional-step
integrator, differentiated with the library's hand-written discrete adjoint
(fsei_adjoint_step) and checkpoint-and-recompute.

Forward: the window starts from (u0, v0, w0) with p = 0 and no Adams-Bashforth
history, applies the body force (fx, fy, fz) at every step, and runs nsteps
steps at a frozen dt (the adjoint of the CFL maximum does not exist).  The
state is checkpointed every `checkpoint_every` steps.  Backward: segments
last to first; each segment is recomputed from its checkpoint (keeping the
per-step inputs) and then walked back step by step with fsei_adjoint_step,
accumulating the force cotangent.  Every step and adjoint step runs in the
library's CUDA kernels; torch only provides memory, the stream and the
autograd plumbing.
"""

import numpy as np
import torch

from . import fsei

STATE = ("u", "v", "w", "p", "hu", "hv", "hw")


def _clone(s):
    out = {k: s[k].clone() for k in STATE}
    out["have_prev_h"] = s["have_prev_h"]
    return out


def frozen_dt(grid, u0, v0, w0, cfl, re, f=None, fconst=(0.0, 0.0, 0.0)):
    """dt that the CFL rule gives for the initial field (one library step on a
    scratch copy; only its dt is kept)."""
    z = torch.zeros_like(u0)
    s = {"u": u0.clone(), "v": v0.clone(), "w": w0.clone(), "p": z.clone(), "hu": z.clone(),
         "hv": z.clone(), "hw": z.clone(), "have_prev_h": 0}
    st = fsei.step(grid, s, f, re=re, dt=0.0, cfl=cfl, fconst=fconst, nsteps=1)
    return st["dt_used"]


class StepWindow(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, v0, w0, fx, fy, fz, grid, nsteps, dt, re, checkpoint_every, fconst):
        f = (fx, fy, fz)
        z = torch.zeros_like(u0)
        s = {"u": u0.detach().clone(), "v": v0.detach().clone(), "w": w0.detach().clone(),
             "p": z.clone(), "hu": z.clone(), "hv": z.clone(), "hw": z.clone(), "have_prev_h": 0}
        ckpts = []
        for n in range(nsteps):
            if n % checkpoint_every == 0:
                ckpts.append((n, _clone(s)))
            fsei.step(grid, s, tuple(t.detach() for t in f), re=re, dt=dt, cfl=0.0,
                      fconst=fconst, nsteps=1, stats=False)
        ctx.grid = grid
        ctx.nsteps = nsteps
        ctx.dt = dt
        ctx.re = re
        ctx.ck = checkpoint_every
        ctx.fconst = fconst
        ctx.ckpts = ckpts
        ctx.f = tuple(t.detach() for t in f)
        return s["u"], s["v"], s["w"]

    @staticmethod
    def backward(ctx, gu, gv, gw):
        grid, dt, re = ctx.grid, ctx.dt, ctx.re
        z = torch.zeros_like(gu)
        adj = {"u": gu.contiguous().clone(), "v": gv.contiguous().clone(),
               "w": gw.contiguous().clone(), "p": z.clone(), "hu": z.clone(), "hv": z.clone(),
               "hw": z.clone()}
        fbar = (z.clone(), z.clone(), z.clone())
        for n0, ck in reversed(ctx.ckpts):
            n1 = min(n0 + ctx.ck, ctx.nsteps)
            s = _clone(ck)
            inputs = []
            for _ in range(n0, n1):
                inputs.append({"u": s["u"].clone(), "v": s["v"].clone(), "w": s["w"].clone(),
                               "have_prev_h": s["have_prev_h"]})
                fsei.step(grid, s, ctx.f, re=re, dt=dt, cfl=0.0, fconst=ctx.fconst, nsteps=1,
                          stats=False)
            for fwd in reversed(inputs):
                fsei.adjoint_step(grid, fwd, adj, fbar, re=re, dt=dt, fconst=ctx.fconst)
        return (adj["u"], adj["v"], adj["w"], fbar[0], fbar[1], fbar[2],
                None, None, None, None, None, None)


def window(grid, u0, v0, w0, fx, fy, fz, nsteps, dt, re, checkpoint_every=5,
           fconst=(0.0, 0.0, 0.0)):
    """(u, v, w) after nsteps steps; differentiable in u0, v0, w0, fx, fy, fz."""
    return StepWindow.apply(u0, v0, w0, fx, fy, fz, grid, nsteps, dt, re, checkpoint_every,
                            tuple(fconst))


def kinetic_energy_subbox(u, v, w, zfaces, lx, ly, half=16):
    """J = 1/2 sum of component^2 times the local volume over the staggered
    points whose cell index lies in the central (2 half)^3 block (dx dy dz_k
    for u and v, dx dy hc_k for w; hc_k the centre-to-centre spacing, half a
    cell at the bottom wall).  A differentiable torch expression of the
    window's output, for gradient runs."""
    nz, ny, nx = u.shape
    zf = np.asarray(zfaces, dtype=np.float64)
    dz = zf[1:] - zf[:-1]
    zc = 0.5 * (zf[1:] + zf[:-1])
    hc = np.empty(nz)
    hc[1:] = zc[1:] - zc[:-1]
    hc[0] = 0.5 * dz[0]
    dx, dy = lx / nx, ly / ny
    k0, j0, i0 = nz // 2 - half, ny // 2 - half, nx // 2 - half
    sl = (slice(k0, k0 + 2 * half), slice(j0, j0 + 2 * half), slice(i0, i0 + 2 * half))
    vu = torch.tensor(dx * dy * dz[sl[0]], dtype=u.dtype, device=u.device)[:, None, None]
    vw = torch.tensor(dx * dy * hc[sl[0]], dtype=u.dtype, device=u.device)[:, None, None]
    return 0.5 * ((u[sl] ** 2 * vu).sum() + (v[sl] ** 2 * vu).sum() + (w[sl] ** 2 * vw).sum())
