"""GPU parity of the discrete adjoint (fsei_adjoint_step, through the C ABI)
against the oracle's adjoint (itself pinned by dot-product identities), and
gradients of a kinetic-energy functional through the checkpointed autograd
window against central finite differences (FP64)."""

import numpy as np
import pytest

from oracle.grid import Grid as OGrid, Z_PERIODIC, Z_WALLS
from oracle import adjoint as oadj
from paper_2103_15187_gb300 import inputs

import parity_util as pu

pytestmark = pytest.mark.gpu

KEYS = ("u", "v", "w", "p", "hu", "hv", "hw")


@pytest.fixture(scope="module")
def fsei():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_15187_gb300 import fsei as mod
    mod.load()
    return mod


@pytest.mark.parametrize("zbc,shape", [(Z_WALLS, (24, 12, 18)), (Z_PERIODIC, (16, 8, 12)),
                                       (Z_WALLS, (48, 36, 17))])
@pytest.mark.parametrize("have_prev", [0, 1])
def test_adjoint_step_matches_oracle(fsei, zbc, shape, have_prev):
    import torch
    nx, ny, nz = shape
    g = OGrid(nx, ny, nz, 2.0, 1.5, zbc, lz=1.7, stretch=2.0)
    rng = np.random.default_rng(nx + have_prev)
    fwd = {k: rng.standard_normal(g.shape) for k in ("u", "v", "w")}
    cot = {k: rng.standard_normal(g.shape) for k in KEYS}
    if zbc == Z_WALLS:
        fwd["w"][0] = 0.0
        for k in ("w", "hw"):
            cot[k][0] = 0.0
    fwd["have_prev_h"] = have_prev
    re, dt = 80.0, 4e-3
    ref = oadj.oracle_adjoint_step(g, fwd, cot, re=re, dt=dt)
    grid = fsei.Grid(nx, ny, nz, 2.0, 1.5, zbc=zbc, lz=1.7, stretch=2.0, prec=fsei.FSEI_FP64)
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")  # noqa: E731
    f = {k: dev(fwd[k]) for k in ("u", "v", "w")}
    f["have_prev_h"] = have_prev
    adj = {k: dev(cot[k]) for k in KEYS}
    fbar = tuple(torch.zeros(g.shape, dtype=torch.float64, device="cuda") for _ in range(3))
    fsei.adjoint_step(grid, f, adj, fbar, re=re, dt=dt)
    torch.cuda.synchronize()
    errs = {k: pu.rel_l2(adj[k].cpu().numpy(), ref[k]) for k in KEYS}
    for name, t in zip(("fx", "fy", "fz"), fbar):
        errs[name] = pu.rel_l2(t.cpu().numpy(), ref[name])
    bad = {k: e for k, e in errs.items() if not e <= 1e-12}
    assert not bad, errs


def _ke_subbox(torch, u, v, w, case, half=16):
    """J = 1/2 sum over staggered points whose cell index lies in the central
    (2 half)^3 block of component^2 times its volume (dz_k for u, v; hc_k
    for w)."""
    zf = inputs.z_faces(case.nz, case.zbc, case.lz, case.stretch)
    dz = zf[1:] - zf[:-1]
    zc = 0.5 * (zf[1:] + zf[:-1])
    hc = np.empty(case.nz)
    hc[1:] = zc[1:] - zc[:-1]
    hc[0] = 0.5 * dz[0]
    dx, dy = case.lx / case.nx, case.ly / case.ny
    k0, j0, i0 = case.nz // 2 - half, case.ny // 2 - half, case.nx // 2 - half
    sl = (slice(k0, k0 + 2 * half), slice(j0, j0 + 2 * half), slice(i0, i0 + 2 * half))
    vu = torch.tensor(dx * dy * dz[sl[0]], dtype=u.dtype, device=u.device)[:, None, None]
    vw = torch.tensor(dx * dy * hc[sl[0]], dtype=u.dtype, device=u.device)[:, None, None]
    return 0.5 * ((u[sl] ** 2 * vu).sum() + (v[sl] ** 2 * vu).sum() + (w[sl] ** 2 * vw).sum())


def _window_case(shape):
    nx, ny, nz = shape
    return inputs.case_channel(nx, ny, nz, steps=20, seed=4)


@pytest.mark.parametrize("shape", [(64, 48, 40), (128, 128, 192)])
def test_window_gradient_matches_finite_differences(fsei, shape):
    """FP64, 20 steps, checkpoint every 5, dt frozen from CFL 0.5 at step 0;
    16 seeded Gaussian directions over (u0, v0, w0, fx, fy, fz), each scaled
    to the norm of the initial velocity so that the step 1e-4 is relative;
    central differences agree with the adjoint to 1e-6.  (With unit-norm
    directions over ~1e7 values each point moves by ~1e-8 and round-off in
    J dominates the difference quotient.)"""
    import torch
    from paper_2103_15187_gb300 import autograd as fad
    case = _window_case(shape)
    grid = pu.gpu_grid(case, fsei.FSEI_FP64)
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")  # noqa: E731
    x0 = [dev(case.u), dev(case.v), dev(case.w)] + [torch.zeros_like(dev(case.u)) for _ in range(3)]
    dt = fad.frozen_dt(grid, x0[0], x0[1], x0[2], case.cfl, case.re, fconst=case.fconst)

    def J(xs):
        u, v, w = fad.window(grid, *xs, nsteps=20, dt=dt, re=case.re, checkpoint_every=5,
                             fconst=case.fconst)
        return _ke_subbox(torch, u, v, w, case)

    xs = [t.clone().requires_grad_(True) for t in x0]
    Jv = J(xs)
    Jv.backward()
    grads = [t.grad.detach() for t in xs]
    for gr in (grads[2], grads[5]):
        assert float(gr[0].abs().max()) == 0.0       # wall face is not an input
    worst = 0.0
    for seed in range(100, 116):
        rng = np.random.default_rng(seed)
        d = [rng.standard_normal(case.u.shape) for _ in range(6)]
        d[2][0] = 0.0
        d[5][0] = 0.0
        nrm = np.sqrt(sum((a * a).sum() for a in d))
        scale = np.sqrt((case.u ** 2).sum() + (case.v ** 2).sum() + (case.w ** 2).sum()) / nrm
        d = [dev(a * scale) for a in d]
        eps = 1e-4
        with torch.no_grad():
            jp = float(J([a + eps * b for a, b in zip(x0, d)]))
            jm = float(J([a - eps * b for a, b in zip(x0, d)]))
        fd = (jp - jm) / (2 * eps)
        ad = float(sum((a * b).sum() for a, b in zip(grads, d)))
        rel = abs(fd - ad) / max(abs(fd), 1e-300)
        worst = max(worst, rel)
    assert worst <= 1e-6, worst


def test_mixed_adjoint_against_fp64_adjoint(fsei):
    """FP32 forward and adjoint (FP64 near-zero Poisson modes) on the same
    window: gradient relative L2 error against the FP64 adjoint, stated."""
    import torch
    from paper_2103_15187_gb300 import autograd as fad
    case = _window_case((64, 48, 40))
    out = {}
    for name, prec, dtype in (("fp64", fsei.FSEI_FP64, torch.float64),
                              ("mixed", fsei.FSEI_MIXED, torch.float32)):
        grid = pu.gpu_grid(case, prec)
        xs = [torch.tensor(a, dtype=dtype, device="cuda").requires_grad_(True)
              for a in (case.u, case.v, case.w)]
        fs = [torch.zeros_like(xs[0]).requires_grad_(True) for _ in range(3)]
        dt = fad.frozen_dt(pu.gpu_grid(case, fsei.FSEI_FP64),
                           *[torch.tensor(a, dtype=torch.float64, device="cuda")
                             for a in (case.u, case.v, case.w)], case.cfl, case.re,
                           fconst=case.fconst)
        u, v, w = fad.window(grid, *xs, *fs, nsteps=20, dt=dt, re=case.re, checkpoint_every=5,
                             fconst=case.fconst)
        _ke_subbox(torch, u, v, w, case).backward()
        out[name] = [t.grad.double() for t in xs + fs]
    num = sum(float(torch.linalg.vector_norm(a - b) ** 2) for a, b in zip(out["mixed"], out["fp64"]))
    den = sum(float(torch.linalg.vector_norm(b) ** 2) for b in out["fp64"])
    err = (num / den) ** 0.5
    print("mixed-vs-fp64 adjoint gradient rel L2: %.3e" % err)
    assert err <= 1e-3, err
