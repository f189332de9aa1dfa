"""GPU parity of the immersed-boundary operators (fsei_ib_forcing,
fsei_ib_loads through the C ABI; Sec. 2.1 Eqs. 4-7, Sec. 3.2) against the
oracle on the same seeded fields and synthetic surfaces (triangulated
spheres standing in for the heart's wet surfaces): forces, interpolated
velocities and loads to 1e-12 in FP64, a few float roundings in mixed
precision; markers too close to a wall skipped and counted as the oracle
rejects them; the forcing driving fractional steps against the oracle doing
the same."""

import numpy as np
import pytest

from oracle.grid import Grid as OGrid, Z_PERIODIC, Z_WALLS
from oracle import ib as oib
from oracle.step import oracle_step
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


def _dev(a, dtype):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _markers(g, seed, n=60, zlim=0.75):
    """A sphere of markers (rotating and translating) plus random ones,
    some of them outside the periodic box (wrapped by the library)."""
    s = inputs.ib_surface((0.6 * g.lx, 0.4 * g.ly, 0.1), 0.35, 1, omega=(0.3, -0.8, 1.1),
                          velocity=(0.5, 0.0, -0.2))
    rng = np.random.default_rng(seed)
    xr = np.column_stack([rng.uniform(-0.5 * g.lx, 1.5 * g.lx, n),
                          rng.uniform(-0.5 * g.ly, 1.5 * g.ly, n),
                          rng.uniform(-zlim, zlim, n)])
    xb = np.vstack([s["xf"], xr])
    ub = np.vstack([s["ub"], rng.standard_normal((n, 3))])
    dvb = np.concatenate([s["af"] * g.dx, rng.uniform(0.2, 1.0, n) * g.dx * g.dy * 0.05])
    return xb, ub, dvb


def _wrap(g, xb):
    x = xb.copy()
    x[:, 0] %= g.lx
    x[:, 1] %= g.ly
    return x


@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
@pytest.mark.parametrize("zbc", [Z_WALLS, Z_PERIODIC])
def test_ib_forcing_matches_oracle(fsei, prec_name, zbc):
    import torch
    g = OGrid(24, 24, 28, 2.0, 1.6, zbc, lz=1.8, stretch=1.8 if zbc == Z_WALLS else 0.0)
    prec = fsei.FSEI_FP64 if prec_name == "fp64" else fsei.FSEI_MIXED
    dtype = torch.float64 if prec_name == "fp64" else torch.float32
    grid = fsei.Grid(g.nx, g.ny, g.nz, g.lx, g.ly, zbc=zbc, lz=1.8, stretch=g.stretch, prec=prec)
    rng = np.random.default_rng(40 + zbc)
    u, v, w = (rng.standard_normal(g.shape) for _ in range(3))
    if g.walls:
        w[0] = 0.0
    xb, ub, dvb = _markers(g, 41 + zbc, zlim=0.75 if g.walls else 1.9)
    dt = 2e-3
    vel = [_dev(a, dtype) for a in (u, v, w)]
    f = [torch.zeros_like(vel[0]) for _ in range(3)]
    mk = {"xb": _dev(xb, torch.float64), "ub": _dev(ub, torch.float64),
          "dvb": _dev(dvb, torch.float64)}
    u_at = torch.empty((len(xb), 3), dtype=torch.float64, device="cuda")
    skipped = fsei.ib_forcing(grid, vel, mk, dt, f, u_at)
    assert skipped == 0
    # the oracle sees exactly the values the GPU was given
    vals = [a.double().cpu().numpy() for a in vel]
    (rx, ry, rz), ui = oib.ib_forcing(g, *vals, _wrap(g, xb), ub, dvb, dt)
    tol = 1e-12 if prec_name == "fp64" else 2e-6
    assert np.max(np.abs(u_at.cpu().numpy() - ui)) <= tol * max(1.0, np.abs(ui).max())
    for a, r in zip(f, (rx, ry, rz)):
        assert pu.rel_l2(a.double().cpu().numpy(), r) <= tol


def test_markers_next_to_walls_are_skipped(fsei):
    import torch
    g = OGrid(16, 16, 20, 1.0, 1.0, Z_WALLS, stretch=1.5)
    grid = fsei.Grid(16, 16, 20, 1.0, 1.0, zbc=Z_WALLS, stretch=1.5, prec=fsei.FSEI_FP64)
    z = np.zeros(g.shape)
    xb = np.array([[0.3, 0.3, 0.0], [0.5, 0.5, -0.999], [0.2, 0.7, 0.998], [0.6, 0.1, 0.5]])
    expected = 0
    for x in xb:
        for loc in (oib.U, oib.V, oib.W):
            try:
                oib.support(g, loc, x)
            except ValueError:
                expected += 1
    assert expected >= 2
    vel = [_dev(z, torch.float64) for _ in range(3)]
    f = [torch.zeros_like(vel[0]) for _ in range(3)]
    mk = {"xb": _dev(xb, torch.float64), "ub": _dev(np.ones((4, 3)), torch.float64),
          "dvb": _dev(np.full(4, 1e-3), torch.float64)}
    assert fsei.ib_forcing(grid, vel, mk, 1e-2, f) == expected


@pytest.mark.parametrize("two", [False, True])
def test_ib_loads_match_oracle(fsei, two):
    import torch
    g = OGrid(32, 32, 36, 2.0, 2.0, Z_WALLS, stretch=1.5)
    grid = fsei.Grid(32, 32, 36, 2.0, 2.0, zbc=Z_WALLS, stretch=1.5, prec=fsei.FSEI_FP64)
    rng = np.random.default_rng(50)
    p, u, v, w = (rng.standard_normal(g.shape) for _ in range(4))
    w[0] = 0.0
    s = inputs.ib_surface((1.0137, 0.9871, 0.05), 0.4, 2, two_sided=two)
    probe, re = 0.06, 80.0
    F, _ = oib.face_loads(g, p, u, v, w, s["xf"], s["nf"], s["af"], s["two_sided"], probe, re)
    Fn = oib.nodal_loads(F, s["tris"], len(s["verts"]))
    surf = {"xf": _dev(s["xf"], torch.float64), "nf": _dev(s["nf"], torch.float64),
            "af": _dev(s["af"], torch.float64),
            "two_sided": _dev(s["two_sided"].astype(np.int32), torch.int32),
            "tris": _dev(s["tris"].astype(np.int32), torch.int32), "nnodes": len(s["verts"])}
    nodal = torch.zeros((len(s["verts"]), 3), dtype=torch.float64, device="cuda")
    ff, sk_faces, sk_nodes = fsei.ib_loads(grid, _dev(p, torch.float64),
                                           [_dev(a, torch.float64) for a in (u, v, w)], surf,
                                           probe, re, node_force=nodal)
    assert sk_faces == 0 and sk_nodes == 0
    assert pu.rel_l2(ff.cpu().numpy(), F) <= 1e-12
    assert pu.rel_l2(nodal.cpu().numpy(), Fn) <= 1e-12


def test_ib_forcing_drives_steps_like_the_oracle(fsei):
    """Three steps of a stretched channel in which every step's body force is
    the IB forcing of a rotating sphere computed from that step's u^n: GPU
    (fsei_ib_forcing into zeroed force fields, then fsei_step) against the
    oracle doing the same, 1e-12 per field."""
    import torch
    case = inputs.case_channel(32, 24, 28, steps=3, kmax=3.0, rms=0.2, seed=60, re=500.0)
    case.cfl, case.dt = 0.0, 1e-3
    g = pu.oracle_grid(case)
    s = inputs.ib_surface((1.3 * np.pi + 0.013, 0.5 * np.pi - 0.021, 0.017), 0.45, 1,
                          omega=(0.0, 0.0, 2.0))
    dvb = s["af"] * g.dx
    grid = pu.gpu_grid(case, fsei.FSEI_FP64)
    st = pu.to_device(pu.initial_state_np(case), torch.float64)
    mk = {"xb": _dev(s["xf"], torch.float64), "ub": _dev(s["ub"], torch.float64),
          "dvb": _dev(dvb, torch.float64)}
    ref = pu.initial_state_np(case)
    prm = pu.params(case)
    for _ in range(3):
        f = [torch.zeros_like(st["u"]) for _ in range(3)]
        assert fsei.ib_forcing(grid, (st["u"], st["v"], st["w"]), mk, case.dt, f) == 0
        fsei.step(grid, st, tuple(f), nsteps=1, **prm)
        fo, _ = oib.ib_forcing(g, ref["u"], ref["v"], ref["w"], s["xf"], s["ub"], dvb, case.dt)
        ref, _ = oracle_step(g, ref, fo, **prm)
    torch.cuda.synchronize()
    got = {k: st[k].cpu().numpy() for k in pu.FIELDS}
    errs = pu.compare(got, ref)
    assert max(errs.values()) <= 1e-12, errs
