"""GPU parity of the third-order Runge-Kutta variant (fsei_step with
scheme FSEI_RK3_CN: three fractional sub-steps per step, Sec. 2.1) against
the oracle's RK3 step on the same seeded inputs: 1e-12 per field in FP64,
1e-5 in velocity for mixed precision; the batch with RK3 boxes equals solo
runs; the adjoint reports the scheme as unsupported."""

import numpy as np
import pytest

from paper_2103_15187_gb300 import inputs

import parity_util as pu

pytestmark = pytest.mark.gpu
RK3 = 1


@pytest.fixture(scope="module")
def fsei():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_15187_gb300 import fsei as mod
    mod.load()
    return mod


def _vel_err(gpu, ref):
    return np.sqrt(sum(np.linalg.norm(gpu[k] - ref[k]) ** 2 for k in "uvw")
                   / sum(np.linalg.norm(ref[k]) ** 2 for k in "uvw"))


def test_rk3_taylor_green_fp64(fsei):
    case = inputs.case_taylor_green(32, steps=5, dt=1e-2)
    gpu, st = pu.run_gpu(case, 5, fsei.FSEI_FP64, scheme=RK3)
    ref, rst = pu.run_oracle(case, 5, scheme=RK3)
    errs = pu.compare(gpu, ref)
    assert max(errs.values()) <= 1e-12, errs
    assert abs(st["dt_used"] - 1e-2) < 1e-17
    assert abs(st["kinetic_energy"] / rst[-1]["kinetic_energy"] - 1) < 1e-12


@pytest.mark.parametrize("shape", [(48, 24, 36), (48, 36, 17)])
def test_rk3_forced_channel_cfl_fp64(fsei, shape):
    """Stretched channel with Gaussian-blob force, Poiseuille drive and CFL
    0.8 (the full step's dt from u^n, shared by the sub-steps); two calls of
    three steps (the second starts from the stored history flag)."""
    nx, ny, nz = shape
    case = inputs.case_channel(nx, ny, nz, steps=6, kmax=4.0, rms=0.3, seed=nx + 1, cfl=0.8,
                               blobs=dict(nblobs=3, sigma=3.0, amp=10.0))
    gpu, st = pu.run_gpu(case, 6, fsei.FSEI_FP64, per_call=3, scheme=RK3)
    ref, rst = pu.run_oracle(case, 6, scheme=RK3)
    errs = pu.compare(gpu, ref)
    assert max(errs.values()) <= 1e-12, errs
    for key in ("dt_used", "cfl", "kinetic_energy"):
        assert abs(st[key] / rst[-1][key] - 1) < 1e-12, (key, st[key], rst[-1][key])


def test_rk3_mixed_channel_50_steps(fsei):
    case = inputs.case_channel(64, 64, 64, steps=50, seed=2, cfl=0.8)
    gpu, _ = pu.run_gpu(case, 50, fsei.FSEI_MIXED, scheme=RK3)
    ref, _ = pu.run_oracle(case, 50, scheme=RK3)
    err = _vel_err(gpu, ref)
    assert err <= 1e-5, (err, pu.compare(gpu, ref))


def test_rk3_batch_equals_solo(fsei):
    import torch
    cases = [inputs.case_taylor_green(16, steps=3, dt=5e-3),
             inputs.case_channel(24, 12, 18, steps=3, seed=30, re=700.0, cfl=0.8)]
    batch = fsei.Batch([dict(nx=c.nx, ny=c.ny, nz=c.nz, lx=c.lx, ly=c.ly, zbc=c.zbc, lz=c.lz,
                             stretch=c.stretch, prec=fsei.FSEI_FP64) for c in cases])
    states = [pu.to_device(pu.initial_state_np(c), torch.float64) for c in cases]
    params = [dict(pu.params(c), scheme=RK3) for c in cases]
    fsei.batch_step(batch, states, None, params, nsteps=3)
    for c, st in zip(cases, states):
        solo, _ = pu.run_gpu(c, 3, fsei.FSEI_FP64, scheme=RK3)
        ref, _ = pu.run_oracle(c, 3, scheme=RK3)
        for k in pu.FIELDS:
            a = st[k].cpu().numpy()
            assert pu.rel_l2(a, solo[k]) <= 1e-13, (c.name, k)
            assert pu.compare({k: a}, ref, fields=(k,))[k] <= 1e-12, (c.name, k)


def test_rk3_adjoint_is_unsupported(fsei):
    import ctypes
    import torch
    g = fsei.Grid(16, 8, 12, 2.0, 1.0, zbc=fsei.FSEI_Z_WALLS, stretch=1.0, prec=fsei.FSEI_FP64)
    z = torch.zeros((12, 8, 16), dtype=torch.float64, device="cuda")
    st = fsei.State(*[ctypes.c_void_p(z.data_ptr())] * 7, 0)
    prm = fsei.StepParams(100.0, 1e-3, 0.0, 1.5, -0.5, (ctypes.c_double * 3)(0, 0, 0), RK3)
    lib = fsei.load()
    r = lib.fsei_adjoint_step(g.handle, ctypes.byref(st), ctypes.byref(prm), ctypes.byref(st),
                              None, None, None, None)
    assert r == 3
