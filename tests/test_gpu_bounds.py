"""Bounds-checking mode (FSEI_CHECK_BOUNDS=1 when a grid is created): every
workspace buffer of the grid sits between guard zones that the library
verifies before each call returns.  Here every entry point that launches
kernels runs in that mode on small ragged grids, with the caller's own
fields guarded the same way by the test (all-ones bytes, a NaN, on both
sides of each field).  A kernel that writes past a buffer's end changes a
guard (FSEI_E_BOUNDS, or a failed check of the caller's guards); one that
reads a guard feeds a NaN into its results, which then miss the oracle or
the unguarded run.  The mode itself must not change what is computed."""

import numpy as np
import pytest

from oracle.grid import Z_PERIODIC, Z_WALLS
from paper_2103_15187_gb300 import inputs

import parity_util as pu

pytestmark = pytest.mark.gpu

GUARD = 16384   # elements of caller-side guard before and after each field


@pytest.fixture(scope="module")
def fsei():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_15187_gb300 import fsei as mod
    mod.load()
    return mod


@pytest.fixture
def checked(monkeypatch):
    monkeypatch.setenv("FSEI_CHECK_BOUNDS", "1")


class Guarded:
    """Device tensors carved out of larger buffers whose margins hold
    all-ones bytes; intact() tells whether every margin is unchanged."""

    def __init__(self):
        self.bufs = []

    def tensor(self, a, dtype):
        import torch
        a = np.ascontiguousarray(a)
        n = a.size
        buf = torch.empty(n + 2 * GUARD, dtype=dtype, device="cuda")
        ints = torch.int64 if dtype == torch.float64 else torch.int32
        buf.view(ints).fill_(-1)
        t = buf[GUARD:GUARD + n].view(a.shape)
        t.copy_(torch.as_tensor(a, dtype=dtype))
        self.bufs.append((buf, ints, n))
        return t

    def state(self, state_np, dtype):
        out = {k: self.tensor(state_np[k], dtype) for k in pu.FIELDS}
        out["have_prev_h"] = state_np.get("have_prev_h", 0)
        return out

    def intact(self):
        for buf, ints, n in self.bufs:
            b = buf.view(ints)
            if not (bool((b[:GUARD] == -1).all()) and bool((b[GUARD + n:] == -1).all())):
                return False
        return True


def _np(state):
    return {k: state[k].double().cpu().numpy() for k in pu.FIELDS}


def test_guard_helper_sees_a_write_past_the_end(fsei):
    import torch
    g = Guarded()
    t = g.tensor(np.zeros((3, 4, 8)), torch.float32)
    assert g.intact()
    g.bufs[0][0][GUARD + t.numel()] = 0.0     # one element past the field
    assert not g.intact()


def test_check_needs_the_mode(fsei, monkeypatch):
    monkeypatch.delenv("FSEI_CHECK_BOUNDS", raising=False)
    grid = fsei.Grid(16, 12, 10, 1.0, 1.0, zbc=fsei.FSEI_Z_WALLS, stretch=1.5)
    with pytest.raises(fsei.FseiError) as ei:
        fsei.check_bounds(grid)
    assert ei.value.status == 3


@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
@pytest.mark.parametrize("which", ["channel", "periodic"])
def test_steps_in_bounds_match_the_oracle(fsei, checked, prec_name, which):
    import torch
    if which == "channel":
        case = inputs.case_channel(48, 36, 17, steps=3, kmax=3.0, rms=0.2, seed=60)
    else:
        case = inputs.case_periodic_random(24, seed=61, steps=3)
    prec = fsei.FSEI_FP64 if prec_name == "fp64" else fsei.FSEI_MIXED
    dtype = torch.float64 if prec_name == "fp64" else torch.float32
    grid = pu.gpu_grid(case, prec)
    gd = Guarded()
    st = gd.state(pu.initial_state_np(case), dtype)
    f = None if case.f is None else tuple(gd.tensor(a, dtype) for a in case.f)
    stats = fsei.step(grid, st, f, nsteps=3, **pu.params(case))
    assert stats["flags"] == 0
    fsei.check_bounds(grid)
    assert gd.intact()
    ref, _ = pu.run_oracle(case, 3)
    errs = pu.compare(_np(st), ref, fields=("u", "v", "w", "p"))
    tol = 1e-12 if prec_name == "fp64" else 1e-5
    assert all(e <= tol for e in errs.values()), errs


@pytest.mark.parametrize("variant", ["rk3", "carreau_yasuda"])
def test_variant_steps_in_bounds_equal_unchecked_runs(fsei, monkeypatch, variant):
    import torch
    case = inputs.case_channel(24, 12, 18, steps=2, kmax=3.0, rms=0.2, seed=62)
    prm = dict(pu.params(case))
    if variant == "rk3":
        prm["scheme"] = fsei.FSEI_RK3_CN
    else:
        prm["rheology"] = dict(eta_inf=0.2, lam=2.0, a=2.0, n=0.5)
    out = []
    for mode in ("0", "1"):
        monkeypatch.setenv("FSEI_CHECK_BOUNDS", mode)
        grid = pu.gpu_grid(case, fsei.FSEI_FP64)
        gd = Guarded()
        st = gd.state(pu.initial_state_np(case), torch.float64)
        fsei.step(grid, st, None, nsteps=2, **prm)
        torch.cuda.synchronize()
        assert gd.intact()
        out.append(_np(st))
        if mode == "1":
            fsei.check_bounds(grid)
    for k in pu.FIELDS:
        assert np.array_equal(out[0][k], out[1][k]), k


@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
def test_poisson_and_adjoint_in_bounds(fsei, monkeypatch, prec_name):
    import torch
    nx, ny, nz = 48, 36, 17
    prec = fsei.FSEI_FP64 if prec_name == "fp64" else fsei.FSEI_MIXED
    dtype = torch.float64 if prec_name == "fp64" else torch.float32
    rng = np.random.default_rng(63)
    zf = inputs.z_faces(nz, Z_WALLS, 1.7, 2.0)
    dz = (zf[1:] - zf[:-1])[:, None, None]
    s = rng.standard_normal((nz, ny, nx))
    s -= (s * dz).sum() / (dz.sum() * nx * ny)
    fwd = {k: rng.standard_normal((nz, ny, nx)) for k in ("u", "v", "w")}
    fwd["w"][0] = 0.0
    cot = {k: rng.standard_normal((nz, ny, nx)) for k in pu.FIELDS}
    cot["w"][0] = 0.0
    cot["hw"][0] = 0.0
    res = []
    for mode in ("0", "1"):
        monkeypatch.setenv("FSEI_CHECK_BOUNDS", mode)
        grid = fsei.Grid(nx, ny, nz, 2.0, 1.5, zbc=Z_WALLS, lz=1.7, stretch=2.0, prec=prec)
        gd = Guarded()
        rhs = gd.tensor(s, dtype)
        phi = gd.tensor(np.zeros_like(s), dtype)
        fsei.poisson_solve(grid, rhs, phi)
        f = {k: gd.tensor(fwd[k], dtype) for k in ("u", "v", "w")}
        f["have_prev_h"] = 1
        adj = {k: gd.tensor(cot[k], dtype) for k in pu.FIELDS}
        fbar = tuple(gd.tensor(np.zeros((nz, ny, nx)), dtype) for _ in range(3))
        fsei.adjoint_step(grid, f, adj, fbar, re=80.0, dt=4e-3)
        torch.cuda.synchronize()
        assert gd.intact()
        if mode == "1":
            fsei.check_bounds(grid)
        res.append([phi.double().cpu().numpy()] + [adj[k].double().cpu().numpy()
                                                    for k in pu.FIELDS]
                   + [t.double().cpu().numpy() for t in fbar])
    for a, b in zip(*res):
        assert np.array_equal(a, b)


def test_ib_forcing_and_loads_in_bounds(fsei, monkeypatch):
    import torch
    nx, ny, nz = 24, 24, 28
    rng = np.random.default_rng(64)
    u, v, w, p = (rng.standard_normal((nz, ny, nx)) for _ in range(4))
    w[0] = 0.0
    s = inputs.ib_surface((1.0, 0.8, 0.05), 0.35, 2, omega=(0.3, -0.8, 1.1),
                          velocity=(0.5, 0.0, -0.2))
    dev = lambda a, dt=torch.float64: torch.tensor(np.ascontiguousarray(a), dtype=dt,  # noqa
                                                   device="cuda")
    res = []
    for mode in ("0", "1"):
        monkeypatch.setenv("FSEI_CHECK_BOUNDS", mode)
        grid = fsei.Grid(nx, ny, nz, 2.0, 1.6, zbc=Z_WALLS, lz=1.8, stretch=1.8,
                         prec=fsei.FSEI_FP64)
        gd = Guarded()
        vel = [gd.tensor(a, torch.float64) for a in (u, v, w)]
        f = [gd.tensor(np.zeros_like(u), torch.float64) for _ in range(3)]
        mk = {"xb": dev(s["xf"]), "ub": dev(s["ub"]), "dvb": dev(s["af"] * 2.0 / nx)}
        u_at = torch.empty((len(s["xf"]), 3), dtype=torch.float64, device="cuda")
        assert fsei.ib_forcing(grid, vel, mk, 2e-3, f, u_at) == 0
        surf = {"xf": dev(s["xf"]), "nf": dev(s["nf"]), "af": dev(s["af"]),
                "two_sided": dev(s["two_sided"].astype(np.int32), torch.int32),
                "tris": dev(s["tris"].astype(np.int32), torch.int32),
                "nnodes": len(s["verts"])}
        ff, sk_f, sk_n = fsei.ib_loads(grid, gd.tensor(p, torch.float64), vel, surf, 0.06, 80.0)
        assert sk_f == 0 and sk_n == 0
        torch.cuda.synchronize()
        assert gd.intact()
        if mode == "1":
            fsei.check_bounds(grid)
        res.append([t.cpu().numpy() for t in f] + [u_at.cpu().numpy(), ff.cpu().numpy()])
    # the spreading adds with atomics: the order of the sums is not fixed
    for a, b in zip(*res):
        assert pu.rel_l2(a, b) <= 1e-13


def test_batch_and_host_state_in_bounds(fsei, checked):
    import torch
    cases = [inputs.case_taylor_green(16, steps=2),
             inputs.case_channel(24, 12, 18, steps=2, kmax=3.0, rms=0.2, seed=65),
             inputs.case_periodic_random(16, seed=66, steps=2)]
    batch = fsei.Batch([dict(nx=c.nx, ny=c.ny, nz=c.nz, lx=c.lx, ly=c.ly, zbc=c.zbc, lz=c.lz,
                             stretch=c.stretch, prec=fsei.FSEI_FP64) for c in cases])
    gd = Guarded()
    states = [gd.state(pu.initial_state_np(c), torch.float64) for c in cases]
    fsei.batch_step(batch, states, None, [pu.params(c) for c in cases], nsteps=2)
    assert gd.intact()
    for c, st in zip(cases, states):
        ref, _ = pu.run_oracle(c, 2)
        errs = pu.compare(_np(st), ref, fields=("u", "v", "w", "p"))
        assert all(e <= 1e-12 for e in errs.values()), errs
    # the state held in host memory, copied through guarded device fields
    case = cases[1]
    grid = pu.gpu_grid(case, fsei.FSEI_FP64)
    host = {k: torch.tensor(v, dtype=torch.float64).pin_memory()
            for k, v in pu.initial_state_np(case).items() if k != "have_prev_h"}
    host["have_prev_h"] = 0
    dev = {k: gd.tensor(np.zeros(host[k].shape), torch.float64) for k in pu.FIELDS}
    fsei.step_host(grid, host, dev, None, nsteps=2, stats=True, **pu.params(case))
    assert gd.intact()
    ref, _ = pu.run_oracle(case, 2)
    errs = pu.compare({k: host[k].numpy() for k in pu.FIELDS}, ref,
                      fields=("u", "v", "w", "p"))
    assert all(e <= 1e-12 for e in errs.values()), errs


@pytest.mark.parametrize("buffer,side,offset", [(0, 0, 0), (5, 1, 0), (9, 1, 4000)])
def test_a_changed_guard_byte_is_reported(fsei, checked, buffer, side, offset):
    """The detector itself: one guard byte changed (inside the library's own
    allocation, by the test hook) is reported by fsei_grid_check_bounds and
    by the next call that launches work, with the buffer, side and
    distance."""
    import torch
    case = inputs.case_channel(24, 12, 18, steps=1, kmax=3.0, rms=0.2, seed=67)
    grid = pu.gpu_grid(case, fsei.FSEI_FP64)
    fsei.check_bounds(grid)
    fsei.poke_guard(grid, buffer, side, offset)
    with pytest.raises(fsei.FseiError) as ei:
        fsei.check_bounds(grid)
    assert ei.value.status == 8, ei.value
    msg = str(ei.value)
    assert ("after" if side else "before") in msg and "buffer %d " % buffer in msg, msg
    assert "%d bytes from" % offset in msg, msg
    st = pu.to_device(pu.initial_state_np(case), torch.float64)
    with pytest.raises(fsei.FseiError) as ei:
        fsei.step(grid, st, None, nsteps=1, **pu.params(case))
    assert ei.value.status == 8, ei.value


def test_poke_guard_rejects_what_does_not_exist(fsei, checked, monkeypatch):
    grid = fsei.Grid(16, 12, 10, 1.0, 1.0, zbc=fsei.FSEI_Z_WALLS, stretch=1.5)
    for args in ((-1, 0, 0), (10 ** 6, 0, 0), (0, 2, 0), (0, 0, 1 << 40)):
        with pytest.raises(fsei.FseiError) as ei:
            fsei.poke_guard(grid, *args)
        assert ei.value.status == 1, (args, ei.value)
    fsei.check_bounds(grid)
    monkeypatch.delenv("FSEI_CHECK_BOUNDS")
    plain = fsei.Grid(16, 12, 10, 1.0, 1.0, zbc=fsei.FSEI_Z_WALLS, stretch=1.5)
    with pytest.raises(fsei.FseiError) as ei:
        fsei.poke_guard(plain, 0, 0, 0)
    assert ei.value.status == 3
