"""fsei_step_host: a state held in host memory advanced through the C ABI
(copies in, the step, copies back on the grid's copy stream) gives exactly
what fsei_step gives on the same state in device memory, call after call
without synchronising in between, with pinned and with pageable host
memory, in both precisions, with forcing, CFL time steps and the RK3
scheme; its statistics are fsei_step's (the kinetic energy, a sum of
per-block atomics, to rounding); NULL or misaligned fields are refused."""

import ctypes

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


def _host_state(case, dtype, pinned):
    import torch
    st = {}
    for k, a in pu.initial_state_np(case).items():
        if k == "have_prev_h":
            st[k] = a
            continue
        t = torch.tensor(a, dtype=dtype)
        st[k] = t.pin_memory() if pinned else t
    return st


@pytest.mark.parametrize("prec_name,pinned,scheme", [("mixed", True, 0), ("mixed", False, 0),
                                                      ("fp64", True, 0), ("fp64", True, 1)])
def test_host_state_steps_equal_device_steps(fsei, prec_name, pinned, scheme):
    import torch
    case = inputs.case_channel(64, 48, 40, steps=4, seed=31, re=700.0,
                               blobs=dict(nblobs=2, sigma=3.0, amp=4.0))
    prec = fsei.FSEI_FP64 if prec_name == "fp64" else fsei.FSEI_MIXED
    dtype = torch.float64 if prec_name == "fp64" else torch.float32
    grid = pu.gpu_grid(case, prec)
    f = pu.force_device(case, dtype)
    prm = dict(pu.params(case), scheme=scheme)
    # device path, one call per step
    ref = pu.to_device(pu.initial_state_np(case), dtype)
    ref_stats = None
    for _ in range(4):
        ref_stats = fsei.step(grid, ref, f, nsteps=1, **prm)
    # host path: three calls without synchronising, the last with stats
    host = _host_state(case, dtype, pinned)
    dev = {k: torch.empty(v.shape, dtype=dtype, device="cuda") for k, v in host.items()
           if k != "have_prev_h"}
    for _ in range(3):
        fsei.step_host(grid, host, dev, f, nsteps=1, stats=False, **prm)
    stats = fsei.step_host(grid, host, dev, f, nsteps=1, stats=True, **prm)
    assert host["have_prev_h"] == 1
    for k in pu.FIELDS:
        assert torch.equal(host[k], ref[k].cpu()), k
    for k in ("dt_used", "cfl", "max_div"):
        assert stats[k] == ref_stats[k], (k, stats[k], ref_stats[k])
    # the kinetic energy is a sum of per-block atomics: equal to rounding
    assert stats["kinetic_energy"] == pytest.approx(ref_stats["kinetic_energy"], rel=1e-12)


def test_join_orders_the_stream_after_the_copies_back(fsei):
    import torch
    case = inputs.case_periodic_random(32, seed=4, steps=2, re=300.0)
    grid = pu.gpu_grid(case, fsei.FSEI_MIXED)
    host = _host_state(case, torch.float32, True)
    dev = {k: torch.empty(v.shape, dtype=torch.float32, device="cuda") for k, v in host.items()
           if k != "have_prev_h"}
    ref = pu.to_device(pu.initial_state_np(case), torch.float32)
    fsei.step(grid, ref, None, nsteps=2, stats=False, **pu.params(case))
    fsei.step_host(grid, host, dev, None, nsteps=2, stats=False, **pu.params(case))
    fsei.step_host_join(grid)
    torch.cuda.current_stream().synchronize()
    for k in pu.FIELDS:
        assert torch.equal(host[k], ref[k].cpu()), k


def test_bad_fields_refused(fsei):
    import torch
    case = inputs.case_periodic_random(16, seed=5, steps=1)
    grid = pu.gpu_grid(case, fsei.FSEI_MIXED)
    lib = fsei.load()
    host = _host_state(case, torch.float32, True)
    dev = {k: torch.zeros(v.numel() + 4, dtype=torch.float32, device="cuda") for k, v in host.items()
           if k != "have_prev_h"}
    prm = fsei.StepParams(100.0, 1e-3, 0.0, 1.5, -0.5, (ctypes.c_double * 3)())

    def st(d, off=0):
        return fsei.State(*[ctypes.c_void_p(d[k].data_ptr() + off) for k in
                            ("u", "v", "w", "p", "hu", "hv", "hw")], 0)
    hs, ds = st(host), st(dev)
    nul = fsei.State(None, None, None, None, None, None, None, 0)
    assert lib.fsei_step_host(grid.handle, ctypes.byref(nul), ctypes.byref(ds), None, None, None,
                              ctypes.byref(prm), 1, None, None) == 1
    assert lib.fsei_step_host(grid.handle, ctypes.byref(hs), ctypes.byref(st(dev, 4)), None,
                              None, None, ctypes.byref(prm), 1, None, None) == 1
