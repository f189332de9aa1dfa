"""Failure reporting of the C ABI, exercised with faults made on the host:
a NaN written into one input value, a fixed time step far above the CFL
limit, a NaN in one box of a batch, and a device-memory budget too small for
a grid.  None of these faults the GPU: the kernels compute on the bad values
and flag them, and the host reads the flags on a synchronising call
(fsei_step_stats.flags and the returned status).  After each fault the same
process steps a healthy state again."""

import os

import numpy as np
import pytest

from paper_2103_15187_gb300 import inputs

import parity_util as pu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fsei():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_15187_gb300 import fsei as mod
    mod.load()
    return mod


def _healthy_step(fsei, prec):
    case = inputs.case_channel(24, 12, 18, steps=2, kmax=3.0, rms=0.2, seed=21)
    gpu, st = pu.run_gpu(case, 2, prec)
    assert st["flags"] == 0 and np.isfinite(gpu["u"]).all()


@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
def test_nan_in_input_reports_nonfinite(fsei, prec_name):
    import torch
    prec = fsei.FSEI_FP64 if prec_name == "fp64" else fsei.FSEI_MIXED
    dtype = torch.float64 if prec_name == "fp64" else torch.float32
    case = inputs.case_channel(24, 12, 18, steps=2, kmax=3.0, rms=0.2, seed=20)
    grid = pu.gpu_grid(case, prec)
    st = pu.to_device(pu.initial_state_np(case), dtype)
    st["u"][5, 3, 7] = float("nan")
    with pytest.raises(fsei.FseiError) as ei:
        fsei.step(grid, st, None, nsteps=2, re=case.re, dt=1e-3, cfl=0.0, fconst=case.fconst)
    assert ei.value.status == 6, ei.value
    assert ei.value.stats["flags"] & fsei.FLAG_NONFINITE
    _healthy_step(fsei, prec)


def test_time_step_above_cfl_limit_reports_cfl(fsei):
    """Taylor-Green at 32^3 with a fixed dt = 0.4: |u_c|/dx + |v_c|/dy peaks
    near |sin(x + y)|/dx = 1/dx (dx = 2 pi / 32), so the new state's CFL
    number is about 2."""
    import torch
    case = inputs.case_taylor_green(32, steps=1)
    grid = pu.gpu_grid(case, fsei.FSEI_FP64)
    st = pu.to_device(pu.initial_state_np(case), torch.float64)
    with pytest.raises(fsei.FseiError) as ei:
        fsei.step(grid, st, None, nsteps=1, re=case.re, dt=0.4, cfl=0.0)
    assert ei.value.status == 7, ei.value
    s = ei.value.stats
    assert s["flags"] & fsei.FLAG_CFL and not s["flags"] & fsei.FLAG_NONFINITE
    assert 1.0 < s["cfl"] < 4.0
    # the same state at a tenth of that dt is accepted
    st = pu.to_device(pu.initial_state_np(case), torch.float64)
    out = fsei.step(grid, st, None, nsteps=1, re=case.re, dt=0.04, cfl=0.0)
    assert out["flags"] == 0 and out["cfl"] < 1.0


def test_nan_in_one_batch_box_is_attributed_to_it(fsei):
    import torch
    cases = [inputs.case_taylor_green(16, steps=2),
             inputs.case_channel(24, 12, 18, steps=2, kmax=3.0, rms=0.2, seed=22),
             inputs.case_periodic_random(16, seed=23, steps=2)]
    batch = fsei.Batch([dict(nx=c.nx, ny=c.ny, nz=c.nz, lx=c.lx, ly=c.ly, zbc=c.zbc, lz=c.lz,
                             stretch=c.stretch, prec=fsei.FSEI_FP64) for c in cases])
    states = [pu.to_device(pu.initial_state_np(c), torch.float64) for c in cases]
    states[1]["w"][4, 2, 3] = float("inf")
    params = [dict(re=c.re, dt=1e-3, cfl=0.0, fconst=c.fconst) for c in cases]
    with pytest.raises(fsei.FseiError) as ei:
        fsei.batch_step(batch, states, None, params, nsteps=2)
    assert ei.value.status == 6 and "box 1" in str(ei.value)
    flags = [s["flags"] for s in ei.value.stats]
    assert flags[1] & fsei.FLAG_NONFINITE and flags[0] == 0 and flags[2] == 0


def test_workspace_budget_reports_nomem(fsei, monkeypatch):
    """FSEI_WORKSPACE_LIMIT_BYTES caps a grid's device allocations: 1 MB is
    too small for a 64^3 grid (FSEI_E_NOMEM, nothing leaked: the same grid is
    created right after without the cap), while a cap above the grid's own
    workspace lets it through."""
    g = fsei.Grid(64, 64, 64, 2 * np.pi, np.pi, zbc=fsei.FSEI_Z_WALLS, stretch=2.0,
                  prec=fsei.FSEI_MIXED)
    need = g.workspace_bytes()
    g.close()
    monkeypatch.setenv("FSEI_WORKSPACE_LIMIT_BYTES", str(1 << 20))
    with pytest.raises(fsei.FseiError) as ei:
        fsei.Grid(64, 64, 64, 2 * np.pi, np.pi, zbc=fsei.FSEI_Z_WALLS, stretch=2.0,
                  prec=fsei.FSEI_MIXED)
    assert ei.value.status == 4, ei.value
    monkeypatch.setenv("FSEI_WORKSPACE_LIMIT_BYTES", str(need))
    g = fsei.Grid(64, 64, 64, 2 * np.pi, np.pi, zbc=fsei.FSEI_Z_WALLS, stretch=2.0,
                  prec=fsei.FSEI_MIXED)
    assert g.workspace_bytes() == need
    g.close()
    monkeypatch.delenv("FSEI_WORKSPACE_LIMIT_BYTES")
    assert "FSEI_WORKSPACE_LIMIT_BYTES" not in os.environ
    _healthy_step(fsei, fsei.FSEI_MIXED)
