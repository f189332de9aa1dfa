"""Helpers shared by the GPU parity tests: run a synthetic case through the
C-ABI library (via the ctypes binding) and through the FP64 oracle on the
same seeded inputs, and compare field by field."""

import numpy as np

from oracle.grid import Grid as OGrid
from oracle.step import oracle_step, oracle_step_rk3

FIELDS = ("u", "v", "w", "p", "hu", "hv", "hw")


def oracle_grid(case):
    return OGrid(case.nx, case.ny, case.nz, case.lx, case.ly, case.zbc, lz=case.lz,
                 stretch=case.stretch)


def initial_state_np(case):
    z = np.zeros_like(case.u)
    return {"u": case.u.copy(), "v": case.v.copy(), "w": case.w.copy(),
            "p": case.p.copy(), "hu": z.copy(), "hv": z.copy(), "hw": z.copy(),
            "have_prev_h": 0}


def params(case):
    return dict(re=case.re, dt=case.dt, cfl=case.cfl, fconst=case.fconst)


def run_oracle(case, nsteps, state=None, scheme=0):
    """nsteps oracle steps: Eq. 3 (scheme 0) or the RK3 variant (scheme 1)."""
    g = oracle_grid(case)
    s = initial_state_np(case) if state is None else state
    stats = []
    for _ in range(nsteps):
        if scheme == 1:
            s, st = oracle_step_rk3(g, s, case.f, **params(case))
        else:
            s, st = oracle_step(g, s, case.f, **params(case))
        stats.append(st)
    return s, stats


def gpu_grid(case, prec, **kw):
    from paper_2103_15187_gb300 import fsei
    return fsei.Grid(case.nx, case.ny, case.nz, case.lx, case.ly, zbc=case.zbc,
                     lz=case.lz, stretch=case.stretch, prec=prec, **kw)


def to_device(state_np, dtype):
    import torch
    out = {k: torch.tensor(state_np[k], dtype=dtype, device="cuda").contiguous()
           for k in FIELDS}
    out["have_prev_h"] = state_np.get("have_prev_h", 0)
    return out


def force_device(case, dtype):
    import torch
    if case.f is None:
        return None
    return tuple(torch.tensor(a, dtype=dtype, device="cuda").contiguous() for a in case.f)


def run_gpu(case, nsteps, prec, grid=None, per_call=None, scheme=0):
    """Advance the case nsteps on the GPU; returns (numpy state, last stats).
    per_call: steps per fsei_step call (default: all in one call); scheme:
    0 Adams-Bashforth (Eq. 3), 1 the RK3 variant."""
    import torch
    from paper_2103_15187_gb300 import fsei
    dtype = torch.float64 if prec == fsei.FSEI_FP64 else torch.float32
    g = grid if grid is not None else gpu_grid(case, prec)
    st = to_device(initial_state_np(case), dtype)
    f = force_device(case, dtype)
    per_call = per_call or nsteps
    stats = None
    done = 0
    while done < nsteps:
        n = min(per_call, nsteps - done)
        stats = fsei.step(g, st, f, nsteps=n, scheme=scheme, **params(case))
        done += n
    torch.cuda.synchronize()
    out = {k: st[k].double().cpu().numpy() for k in FIELDS}
    return out, stats


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def rel_l2_mean_free(a, b):
    return rel_l2(a - a.mean(), b - b.mean())


def compare(gpu, ref, fields=FIELDS):
    """Relative L2 error per field (pressure with its mean removed)."""
    out = {}
    for k in fields:
        if k == "p":
            out[k] = rel_l2_mean_free(gpu[k], ref[k])
        else:
            out[k] = rel_l2(gpu[k], ref[k])
    return out
