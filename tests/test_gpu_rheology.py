"""GPU parity of the Carreau-Yasuda (shear-thinning) step (fsei_step with
rheology = FSEI_CARREAU_YASUDA, Sec. 2.1) against the oracle's step with
the same law on the same seeded inputs: 1e-12 per field in FP64 across the
Euler start and Adams-Bashforth steps, 1e-5 in velocity for mixed
precision; a batch with shear-thinning boxes against the oracle; the law
refused with the RK3 scheme and in the adjoint."""

import ctypes

import numpy as np
import pytest

from oracle.step import oracle_step
from paper_2103_15187_gb300 import inputs

import parity_util as pu

pytestmark = pytest.mark.gpu

CY = dict(lam=1.5, n=0.5, a=2.0, eta_inf=0.3)


@pytest.fixture(scope="module")
def fsei():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_15187_gb300 import fsei as mod
    mod.load()
    return mod


def _oracle(case, nsteps, cy=CY):
    g = pu.oracle_grid(case)
    s = pu.initial_state_np(case)
    for _ in range(nsteps):
        s, _ = oracle_step(g, s, case.f, rheology=cy, **pu.params(case))
    return s


def _gpu(fsei, case, nsteps, prec, per_call=None, cy=CY):
    import torch
    dtype = torch.float64 if prec == fsei.FSEI_FP64 else torch.float32
    grid = pu.gpu_grid(case, prec)
    st = pu.to_device(pu.initial_state_np(case), dtype)
    f = pu.force_device(case, dtype)
    done = 0
    per_call = per_call or nsteps
    while done < nsteps:
        n = min(per_call, nsteps - done)
        fsei.step(grid, st, f, nsteps=n, rheology=cy, **pu.params(case))
        done += n
    torch.cuda.synchronize()
    return {k: st[k].double().cpu().numpy() for k in pu.FIELDS}


@pytest.mark.parametrize("shape", [(48, 24, 36), (32, 36, 17)])
def test_shear_thinning_channel_fp64(fsei, shape):
    """Stretched channel with force blobs and CFL time steps; five steps in
    calls of two (the stored history carries the non-Newtonian term)."""
    nx, ny, nz = shape
    case = inputs.case_channel(nx, ny, nz, steps=5, kmax=4.0, rms=0.4, seed=nx + 3, re=150.0,
                               blobs=dict(nblobs=3, sigma=3.0, amp=5.0))
    gpu = _gpu(fsei, case, 5, fsei.FSEI_FP64, per_call=2)
    ref = _oracle(case, 5)
    errs = pu.compare(gpu, ref)
    assert max(errs.values()) <= 1e-12, errs


def test_shear_thinning_periodic_box_fp64(fsei):
    case = inputs.case_periodic_random(24, seed=9, steps=4, re=80.0)
    gpu = _gpu(fsei, case, 4, fsei.FSEI_FP64)
    ref = _oracle(case, 4)
    errs = pu.compare(gpu, ref)
    assert max(errs.values()) <= 1e-12, errs


def test_shear_thinning_mixed_channel(fsei):
    case = inputs.case_channel(64, 64, 48, steps=20, kmax=4.0, rms=0.3, seed=7, re=300.0)
    gpu = _gpu(fsei, case, 20, fsei.FSEI_MIXED)
    ref = _oracle(case, 20)
    vel = np.sqrt(sum(np.linalg.norm(gpu[k] - ref[k]) ** 2 for k in "uvw")
                  / sum(np.linalg.norm(ref[k]) ** 2 for k in "uvw"))
    print("mixed Carreau-Yasuda channel, 20 steps: velocity rel L2 %.3e" % vel)
    assert vel <= 1e-5, vel


def test_shear_thinning_batch(fsei):
    import torch
    cases = [inputs.case_channel(24, 12, 18, steps=3, seed=70, re=120.0),
             inputs.case_channel(24, 12, 18, steps=3, seed=71, re=90.0),
             inputs.case_periodic_random(16, seed=72, steps=3, re=60.0)]
    batch = fsei.Batch([dict(nx=c.nx, ny=c.ny, nz=c.nz, lx=c.lx, ly=c.ly, zbc=c.zbc, lz=c.lz,
                             stretch=c.stretch, prec=fsei.FSEI_FP64) for c in cases])
    states = [pu.to_device(pu.initial_state_np(c), torch.float64) for c in cases]
    params = [dict(pu.params(c), rheology=CY) for c in cases]
    fsei.batch_step(batch, states, None, params, nsteps=3)
    for c, st in zip(cases, states):
        ref = _oracle(c, 3)
        got = {k: st[k].cpu().numpy() for k in pu.FIELDS}
        errs = pu.compare(got, ref)
        assert max(errs.values()) <= 1e-12, (c.name, errs)


def test_shear_thinning_refused_with_rk3_and_in_the_adjoint(fsei):
    import torch
    case = inputs.case_channel(24, 12, 18, steps=1, seed=73)
    grid = pu.gpu_grid(case, fsei.FSEI_FP64)
    st = pu.to_device(pu.initial_state_np(case), torch.float64)
    with pytest.raises(fsei.FseiError) as ei:
        fsei.step(grid, st, None, nsteps=1, scheme=fsei.FSEI_RK3_CN, rheology=CY,
                  **pu.params(case))
    assert ei.value.status == 3
    z = torch.zeros_like(st["u"])
    s = fsei.State(*[ctypes.c_void_p(z.data_ptr())] * 7, 0)
    rh, cy = fsei._rheology(CY)
    prm = fsei.StepParams(100.0, 1e-3, 0.0, 1.5, -0.5, (ctypes.c_double * 3)(0, 0, 0), 0, rh, cy)
    lib = fsei.load()
    assert lib.fsei_adjoint_step(grid.handle, ctypes.byref(s), ctypes.byref(prm),
                                 ctypes.byref(s), None, None, None, None) == 3
