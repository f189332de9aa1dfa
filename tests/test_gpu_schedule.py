"""Launch schedules and their autotuner (fsei_grid_autotune,
fsei_grid_get_schedule, fsei_grid_set_schedule, fsei_batch_autotune).

A schedule fixes tile shapes and solver splits only: every admissible value
of every field must give the step at parity with the oracle (1e-12 per field
in FP64, 1e-5 in velocity for mixed precision), inadmissible values must be
refused with FSEI_E_ARG, and the autotuner must pick an admissible schedule,
remember it for later grids of the shape, and leave the caller's timing sums
alone."""

import numpy as np
import pytest

from paper_2103_15187_gb300 import inputs

import parity_util as pu

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_VEL_TOL = 1e-5

# values tried per field: the admissible ones and some that never are
TRIALS = {
    "rhs_cells_per_lane": [4, 8, 2, 5, 16, 6, 3],
    "rhs_march": [(4, 4), (4, 8), (8, 4), (2, 4), (4, 3)],
    "poisson": [(16, 16), (32, 8), (16, 8), (8, 32), (64, 4)],
    "rfft_rows_per_block": [1, 2, 4, 8, 16, 3, 32],
    "ffty_columns_per_block": [2, 4, 8, 16, 32, 3, 64],
    "project_passes_per_thread": [1, 2, 4, 8, 3, 16],
    "zsweep_columns_per_lane": [1, 2, 3, 4],
}


@pytest.fixture(scope="module")
def fsei():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_15187_gb300 import fsei as mod
    mod.load()
    return mod


@pytest.fixture(scope="module")
def channel():
    # nz = 256 admits two Poisson splits in single precision; ny = 32 several
    # y-transform widths and x-transform row counts; nx = 64 both RHS widths
    case = inputs.case_channel(64, 32, 256, steps=2, seed=21, re=1500.0)
    ref, _ = pu.run_oracle(case, 2)
    return case, ref


def _check(fsei, prec, gpu, ref):
    if prec == fsei.FSEI_FP64:
        errs = pu.compare(gpu, ref)
        assert all(e <= FP64_TOL for e in errs.values()), errs
    else:
        vel = np.sqrt(sum(np.linalg.norm(gpu[k] - ref[k]) ** 2 for k in "uvw")
                      / sum(np.linalg.norm(ref[k]) ** 2 for k in "uvw"))
        assert vel <= MIXED_VEL_TOL, vel


def _variants(key, value):
    if key == "poisson":
        return {"poisson_lanes_per_line": value[0], "poisson_rows_per_lane": value[1]}
    if key == "rhs_march":
        return {"rhs_cells_per_lane": value[0], "rhs_rows_per_strip": value[1]}
    return {key: value}


@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
@pytest.mark.parametrize("key", sorted(TRIALS))
def test_every_admissible_schedule_at_parity(fsei, channel, prec_name, key):
    case, ref = channel
    prec = fsei.FSEI_FP64 if prec_name == "fp64" else fsei.FSEI_MIXED
    admitted = []
    for value in TRIALS[key]:
        grid = pu.gpu_grid(case, prec)
        base = grid.schedule
        try:
            grid.set_schedule(_variants(key, value))
        except fsei.FseiError as exc:
            assert exc.status == 1, exc        # FSEI_E_ARG
            assert grid.schedule == base       # a refused schedule changes nothing
            continue
        admitted.append(value)
        got = grid.schedule
        for k, v in _variants(key, value).items():
            assert got[k] == v
        gpu, _ = pu.run_gpu(case, 2, prec, grid=grid)
        _check(fsei, prec, gpu, ref)
    # the values that are never admissible stayed out; the fields with
    # choices on this grid offered at least two
    # (strips of 8 need ny = 64 with 8 rows per block; 8 cells per lane leave
    # 8 lanes per row; 2 floats are 8 bytes per lane)
    never = {"rhs_cells_per_lane": [5, 16, 6, 3], "rhs_march": [(4, 8), (8, 4), (2, 4), (4, 3)],
             "poisson": [(16, 8), (8, 32), (64, 4)],
             "rfft_rows_per_block": [3, 32], "ffty_columns_per_block": [3, 64],
             "project_passes_per_thread": [3, 16],
             "zsweep_columns_per_lane": [3, 4]}[key]
    assert not set(admitted) & set(never), admitted
    multi = {"rhs_cells_per_lane": prec_name == "mixed", "rhs_march": False,
             "poisson": prec_name == "mixed",
             "rfft_rows_per_block": True, "ffty_columns_per_block": True,
             "project_passes_per_thread": True, "zsweep_columns_per_lane": True}[key]
    assert len(admitted) >= (2 if multi else 1), admitted


@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
def test_autotune_picks_admissible_schedule_and_caches_it(fsei, channel, prec_name):
    case, ref = channel
    prec = fsei.FSEI_FP64 if prec_name == "fp64" else fsei.FSEI_MIXED
    grid = pu.gpu_grid(case, prec)
    # timing sums in progress survive the autotune untouched
    fsei.set_kernel_timing(grid, True)
    gpu0, _ = pu.run_gpu(case, 1, prec, grid=grid)
    tuned = grid.autotune(force=True)
    kt = fsei.kernel_times(grid)
    fsei.set_kernel_timing(grid, False)
    assert kt["rhs_x (RHS + x sweep)"][1] == 1, kt
    assert kt["project (+ p update, stats)"][1] == 1, kt
    assert grid.schedule == tuned
    grid.set_schedule(tuned)                   # admissible by construction
    # a later grid of the shape starts from the tuned schedule; a later
    # autotune without force measures nothing and returns it
    later = pu.gpu_grid(case, prec)
    assert later.schedule == tuned
    assert later.autotune() == tuned
    gpu, _ = pu.run_gpu(case, 2, prec, grid=later)
    _check(fsei, prec, gpu, ref)


def test_batch_autotune_keeps_solo_equality(fsei):
    """After fsei_batch_autotune every box still equals fsei_step on a solo
    grid of its shape (created afterwards: it takes the cached schedule)."""
    import torch
    cases = [inputs.case_channel(64, 32, 256, steps=3, seed=22, re=1200.0),
             inputs.case_taylor_green(32, steps=3)]
    batch = fsei.Batch([dict(nx=c.nx, ny=c.ny, nz=c.nz, lx=c.lx, ly=c.ly, zbc=c.zbc, lz=c.lz,
                             stretch=c.stretch, prec=fsei.FSEI_MIXED) for c in cases])
    batch.autotune(force=True)
    states = [pu.to_device(pu.initial_state_np(c), torch.float32) for c in cases]
    params = [pu.params(c) for c in cases]
    fsei.batch_step(batch, states, None, params, nsteps=3)
    torch.cuda.synchronize()
    for c, st in zip(cases, states):
        solo, _ = pu.run_gpu(c, 3, fsei.FSEI_MIXED)
        for k in pu.FIELDS:
            err = pu.rel_l2(st[k].double().cpu().numpy(), solo[k])
            assert err <= 1e-15, (c.name, k, err)


def test_batch_group_tuning(fsei):
    """Three boxes of one description tuned as their grouped launches (the
    second pass of fsei_batch_autotune): the group's schedule is admissible,
    shared by the three boxes and remembered for the shape, the boxes agree
    with solo grids created afterwards (to single-precision rounding: a
    group of several boxes runs the group entries of the kernels, compiled
    apart from the solo ones), and one of them meets the oracle."""
    import torch
    cases = [inputs.case_channel(64, 32, 48, steps=3, seed=s, re=900.0) for s in (41, 42, 43)]
    cases.append(inputs.case_taylor_green(32, steps=3))
    batch = fsei.Batch([dict(nx=c.nx, ny=c.ny, nz=c.nz, lx=c.lx, ly=c.ly, zbc=c.zbc, lz=c.lz,
                             stretch=c.stretch, prec=fsei.FSEI_MIXED) for c in cases])
    batch.autotune(force=True)
    later = pu.gpu_grid(cases[0], fsei.FSEI_MIXED)
    tuned = later.schedule
    # admissible: the grid accepts it back
    later.set_schedule(tuned)
    states = [pu.to_device(pu.initial_state_np(c), torch.float32) for c in cases]
    params = [pu.params(c) for c in cases]
    fsei.batch_step(batch, states, None, params, nsteps=3)
    torch.cuda.synchronize()
    for c, st in zip(cases, states):
        solo, _ = pu.run_gpu(c, 3, fsei.FSEI_MIXED)
        for k in pu.FIELDS:
            err = pu.rel_l2(st[k].double().cpu().numpy(), solo[k])
            # the pressure carries the Poisson solve's amplification of the
            # low modes: its rounding differences are the largest
            assert err <= (1e-5 if k == "p" else 1e-6), (c.name, k, err)
    ref, _ = pu.run_oracle(cases[1], 3)
    got = {k: states[1][k].double().cpu().numpy() for k in pu.FIELDS}
    _check(fsei, fsei.FSEI_MIXED, got, ref)
