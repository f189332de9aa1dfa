"""Batched ensemble (fsei_batch_step over boxes of uneven sizes, grouped
launches): every box must agree with fsei_step on that box alone to
rounding (1e-13 per field: the grouped kernels are the same bodies compiled
into another entry, so their rounding may differ in the last bits), across
two calls (the second re-captures with the history flags set), and must
meet the FP64 oracle run on that box: 1e-12 per field in FP64, 1e-5 in
velocity for mixed precision."""

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


def _boxes():
    """Eight boxes of five descriptions: three channels of one shape (other
    seeds and Reynolds numbers) and two Taylor-Green boxes of one shape (other
    time steps) share a description, so they are launched together."""
    cases = [inputs.case_taylor_green(32, steps=5),
             inputs.case_periodic_random(16, seed=7, steps=5),
             inputs.case_channel(48, 24, 20, steps=5, seed=8, re=900.0),
             inputs.case_channel(64, 64, 40, steps=5, seed=9, re=3000.0,
                                 blobs=dict(nblobs=3, sigma=3.0, amp=5.0)),
             inputs.case_channel(24, 12, 18, steps=5, seed=10, re=600.0),
             inputs.case_channel(24, 12, 18, steps=5, seed=11, re=1500.0),
             inputs.case_taylor_green(32, steps=5, dt=2e-3),
             inputs.case_channel(24, 12, 18, steps=5, seed=12, re=300.0,
                                 blobs=dict(nblobs=2, sigma=2.0, amp=4.0))]
    return cases


@pytest.mark.parametrize("max_group,groups", [(0, 5), (1, 8), (2, 6)])
@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
def test_batch_equals_solo_runs(fsei, prec_name, max_group, groups):
    import torch
    prec = fsei.FSEI_FP64 if prec_name == "fp64" else fsei.FSEI_MIXED
    dtype = torch.float64 if prec_name == "fp64" else torch.float32
    cases = _boxes()
    batch = fsei.Batch([dict(nx=c.nx, ny=c.ny, nz=c.nz, lx=c.lx, ly=c.ly, zbc=c.zbc, lz=c.lz,
                             stretch=c.stretch, prec=prec) for c in cases])
    batch.set_max_group(max_group)
    states = [pu.to_device(pu.initial_state_np(c), dtype) for c in cases]
    forces = [pu.force_device(c, dtype) for c in cases]
    params = [pu.params(c) for c in cases]
    stats1 = fsei.batch_step(batch, states, forces, params, nsteps=3)
    fsei.batch_step(batch, states, forces, params, nsteps=2)
    assert batch.launch_groups == groups
    assert all(s["max_div"] < (1e-9 if prec_name == "fp64" else 1e-2) for s in stats1)
    torch.cuda.synchronize()
    for c, st in zip(cases, states):
        solo, _ = pu.run_gpu(c, 5, prec)
        got = {k: st[k].double().cpu().numpy() for k in pu.FIELDS}
        for k in pu.FIELDS:
            err = pu.rel_l2(got[k], solo[k])
            assert err <= 1e-13 if prec_name == "fp64" else err <= 1e-6, (c.name, k, err)
        ref, _ = pu.run_oracle(c, 5)
        if prec_name == "fp64":
            errs = pu.compare(got, ref)
            assert max(errs.values()) <= 1e-12, (c.name, errs)
        else:
            vel = np.sqrt(sum(np.linalg.norm(got[k] - ref[k]) ** 2 for k in "uvw")
                          / sum(np.linalg.norm(ref[k]) ** 2 for k in "uvw"))
            assert vel <= 1e-5, (c.name, vel)


def test_ensemble_generator_mix():
    cases = inputs.case_ensemble(nboxes=8, steps=1, sizes=((16, 16, 16), (24, 24, 20)))
    assert len(cases) == 8
    assert {(c.nx, c.ny, c.nz) for c in cases} <= {(16, 16, 16), (24, 24, 20)}
    assert all(500.0 <= c.re <= 4000.0 for c in cases)
