"""GPU parity of the RHS + x sweep marched along y (k_rhs_x_march, chosen by
the schedule field rhs_rows_per_strip) against the oracle's step (Sec. 2.1,
Eq. 3; Sec. 3.1): lines of 16 to 128 lanes (within a warp and across two or
four warps), 16- and 32-byte lanes (4 floats, 8 floats, 4 doubles), walls
and periodic z, first and last strips whose neighbour rows wrap around the
periodic y end, body forces and the Carreau-Yasuda extra term.  1e-12 per
field in FP64, 1e-5 in velocity for mixed precision; and the same step with
the row-resident kernel agrees to rounding."""

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


def _vel_err(gpu, ref):
    return np.sqrt(sum(np.linalg.norm(gpu[k] - ref[k]) ** 2 for k in "uvw")
                   / sum(np.linalg.norm(ref[k]) ** 2 for k in "uvw"))


def _check(fsei, prec, gpu, ref):
    if prec == fsei.FSEI_FP64:
        errs = pu.compare(gpu, ref)
        assert max(errs.values()) <= 1e-12, errs
    else:
        vel = _vel_err(gpu, ref)
        assert vel <= 1e-5, (vel, pu.compare(gpu, ref))


def _run(fsei, case, nsteps, prec, sched, rheology=None):
    import torch
    dtype = torch.float64 if prec == fsei.FSEI_FP64 else torch.float32
    grid = pu.gpu_grid(case, prec)
    grid.set_schedule(sched)
    got = grid.schedule
    for k, v in sched.items():
        assert got[k] == v, (k, got)
    st = pu.to_device(pu.initial_state_np(case), dtype)
    f = pu.force_device(case, dtype)
    kw = dict(rheology=rheology) if rheology else {}
    fsei.step(grid, st, f, nsteps=nsteps, **kw, **pu.params(case))
    torch.cuda.synchronize()
    return {k: st[k].double().cpu().numpy() for k in pu.FIELDS}


def _oracle(case, nsteps, rheology=None):
    if rheology is None:
        return pu.run_oracle(case, nsteps)[0]
    g = pu.oracle_grid(case)
    s = pu.initial_state_np(case)
    for _ in range(nsteps):
        s, _ = oracle_step(g, s, case.f, rheology=rheology, **pu.params(case))
    return s


# (nx, ny, nz, walls, precision, cells per lane, rows per strip)
CASES = [
    (64, 32, 12, True, "mixed", 4, 4),      # 16 lanes, 8 rows per block
    (128, 16, 10, True, "mixed", 4, 4),     # 32 lanes
    (256, 16, 9, True, "mixed", 4, 8),      # 64 lanes (two warps), odd nz
    (256, 32, 8, False, "mixed", 4, 16),    # periodic z
    (512, 24, 8, True, "mixed", 4, 4),      # 128 lanes (four warps), ny = 24
    (256, 16, 8, False, "mixed", 8, 4),     # 8 floats per lane, 32 lanes
    (512, 8, 9, True, "mixed", 8, 4),       # 8 floats per lane, 64 lanes
    (64, 32, 10, True, "fp64", 4, 4),       # 4 doubles per lane
    (256, 16, 8, False, "fp64", 4, 8),
    (512, 8, 8, True, "fp64", 4, 4),
]


@pytest.mark.parametrize("nx,ny,nz,walls,prec_name,cpl,strip", CASES)
def test_marched_rhs_against_oracle(fsei, nx, ny, nz, walls, prec_name, cpl, strip):
    if walls:
        case = inputs.case_channel(nx, ny, nz, steps=3, kmax=4.0, rms=0.3, seed=nx + ny + nz,
                                   re=400.0, blobs=dict(nblobs=2, sigma=2.0, amp=3.0))
    else:
        case = inputs.case_periodic_random(nx, seed=nx + ny, steps=3, re=300.0, ny=ny, nz=nz)
    prec = fsei.FSEI_FP64 if prec_name == "fp64" else fsei.FSEI_MIXED
    sched = {"rhs_cells_per_lane": cpl, "rhs_rows_per_strip": strip}
    gpu = _run(fsei, case, 3, prec, sched)
    _check(fsei, prec, gpu, _oracle(case, 3))
    # the row-resident kernel on the same grid: the same operations per cell
    row = _run(fsei, case, 3, prec, {"rhs_cells_per_lane": cpl, "rhs_rows_per_strip": 0})
    tol = 1e-13 if prec == fsei.FSEI_FP64 else 1e-6
    assert _vel_err(gpu, row) <= tol


@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
def test_marched_rhs_with_shear_thinning_term(fsei, prec_name):
    case = inputs.case_channel(256, 16, 10, steps=3, kmax=4.0, rms=0.3, seed=5, re=200.0)
    prec = fsei.FSEI_FP64 if prec_name == "fp64" else fsei.FSEI_MIXED
    gpu = _run(fsei, case, 3, prec, {"rhs_cells_per_lane": 4, "rhs_rows_per_strip": 8},
               rheology=CY)
    _check(fsei, prec, gpu, _oracle(case, 3, rheology=CY))


def test_strip_lengths_offered(fsei):
    """Strips are offered only where 16 or 32 bytes per lane, 16 to 128
    lanes per row and ny a multiple of the block's rows times the strip
    hold; anything else is refused with FSEI_E_ARG."""
    case = inputs.case_channel(256, 16, 8, steps=1, seed=1)
    grid = pu.gpu_grid(case, fsei.FSEI_MIXED)
    grid.set_schedule({"rhs_cells_per_lane": 4, "rhs_rows_per_strip": 8})   # 2 x 8 = 16
    for bad in ({"rhs_cells_per_lane": 4, "rhs_rows_per_strip": 16},       # 2 x 16 > 16
                {"rhs_cells_per_lane": 2, "rhs_rows_per_strip": 4},        # 8 bytes per lane
                {"rhs_cells_per_lane": 4, "rhs_rows_per_strip": 3},
                {"rhs_cells_per_lane": 4, "rhs_rows_per_strip": 1}):
        with pytest.raises(fsei.FseiError) as ei:
            grid.set_schedule(bad)
        assert ei.value.status == 1
