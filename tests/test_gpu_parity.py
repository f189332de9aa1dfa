"""GPU parity of the CUDA fractional step (through the C ABI) against the FP64
oracle on the same seeded inputs (Sec. 2.1, Eq. 3; Sec. 3.1).

FP64 gate: relative L2 <= 1e-12 per field.  Mixed precision: velocity
relative L2 <= 1e-5 against the FP64 oracle after 100 steps.  Grids include
ragged tiles (extents that are not multiples of the kernels' tile widths),
periodic and wall-bounded z, stretched meshes, body forces and CFL-driven dt.
"""

import numpy as np
import pytest

from paper_2103_15187_gb300 import inputs
from oracle.grid import Grid as OGrid, Z_PERIODIC, Z_WALLS
from oracle.poisson import oracle_poisson, z_poisson_coefficients, modified_wavenumbers
from oracle.tridiag import thomas, cyclic_thomas

import parity_util as pu

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def fsei():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_15187_gb300 import fsei as mod
    mod.load()
    return mod


def _compatible_rhs(g, seed):
    rng = np.random.default_rng(seed)
    s = rng.standard_normal(g.shape)
    vol = g.cell_volume_uvp()
    return s - (s * vol).sum() / (vol.sum() * g.nx * g.ny)


POISSON_GRIDS = [
    (12, 24, 9, Z_WALLS, 2.0),      # ragged: 12/2 = 6 modes, odd nz
    (32, 32, 32, Z_PERIODIC, 0.0),
    (48, 36, 20, Z_WALLS, 2.0),
    (64, 16, 24, Z_PERIODIC, 0.0),
    (96, 96, 40, Z_WALLS, 1.5),     # radix-3 FFT lengths
    (256, 64, 48, Z_WALLS, 2.0),
]


@pytest.mark.parametrize("nx,ny,nz,zbc,stretch", POISSON_GRIDS)
def test_poisson_fp64_matches_oracle(fsei, nx, ny, nz, zbc, stretch):
    import torch
    g = OGrid(nx, ny, nz, 2 * np.pi, np.pi, zbc, lz=2.0, stretch=stretch)
    s = _compatible_rhs(g, nx + ny + nz)
    ref = oracle_poisson(g, s)
    grid = fsei.Grid(nx, ny, nz, 2 * np.pi, np.pi, zbc=zbc, lz=2.0, stretch=stretch,
                     prec=fsei.FSEI_FP64)
    rhs = torch.tensor(s, dtype=torch.float64, device="cuda")
    phi = torch.empty_like(rhs)
    fsei.poisson_solve(grid, rhs, phi)
    torch.cuda.synchronize()
    err = pu.rel_l2(phi.cpu().numpy(), ref)
    assert err <= FP64_TOL, err


@pytest.mark.parametrize("nx,ny,nz,zbc,stretch", POISSON_GRIDS[:4])
def test_poisson_mixed_error_stated(fsei, nx, ny, nz, zbc, stretch):
    import torch
    g = OGrid(nx, ny, nz, 2 * np.pi, np.pi, zbc, lz=2.0, stretch=stretch)
    s = _compatible_rhs(g, 7 + nx)
    ref = oracle_poisson(g, s)
    grid = fsei.Grid(nx, ny, nz, 2 * np.pi, np.pi, zbc=zbc, lz=2.0, stretch=stretch,
                     prec=fsei.FSEI_MIXED)
    rhs = torch.tensor(s, dtype=torch.float32, device="cuda")
    phi = torch.empty_like(rhs)
    fsei.poisson_solve(grid, rhs, phi)
    torch.cuda.synchronize()
    err = pu.rel_l2(phi.double().cpu().numpy(), ref)
    assert err <= 1e-5, err


def _assert_fp64(gpu, ref, tol=FP64_TOL):
    errs = pu.compare(gpu, ref)
    bad = {k: e for k, e in errs.items() if not e <= tol}
    assert not bad, errs


@pytest.mark.parametrize("zbc", [Z_WALLS, Z_PERIODIC])
def test_forced_rest_state_fp64_one_step(fsei, zbc):
    """Fluid at rest driven by a random body force: no advection, so one step
    exercises the sweeps, the Poisson solve and the projection alone."""
    from paper_2103_15187_gb300.inputs import Case
    nx, ny, nz = 24, 12, 18
    rng = np.random.default_rng(11)
    z = np.zeros((nz, ny, nx))
    f = tuple(rng.standard_normal((nz, ny, nx)) for _ in range(3))
    if zbc == Z_WALLS:
        f[2][0] = 0.0
    case = Case("rest", nx, ny, nz, 2.0, 1.0, zbc, 1.5, 2.0, 50.0, 1e-2, 0.0, 1,
                z, z.copy(), z.copy(), z.copy(), f)
    gpu, _ = pu.run_gpu(case, 1, fsei.FSEI_FP64)
    ref, _ = pu.run_oracle(case, 1)
    _assert_fp64(gpu, ref)


@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
def test_strongly_viscous_forced_channel(fsei, prec_name):
    """Re = 0.05 and dt = 1e-2 on a 64-wide box: beta/dx^2 ~ 15, so the
    factorised x solve's recurrence decays slowly (alpha ~ 0.77) and the
    register x solve takes its full cyclic scan of carries instead of the
    few-lane sum used when alpha^4 is below rounding.  Two steps (Euler start,
    then Adams-Bashforth) from rest under a random force, against the oracle:
    1e-12 per field in FP64, 1e-5 in velocity for mixed precision."""
    from paper_2103_15187_gb300.inputs import Case
    nx, ny, nz = 64, 16, 16
    rng = np.random.default_rng(19)
    z = np.zeros((nz, ny, nx))
    f = tuple(rng.standard_normal((nz, ny, nx)) for _ in range(3))
    f[2][0] = 0.0
    case = Case("viscous", nx, ny, nz, 2.0, 1.0, Z_WALLS, 2.0, 2.0, 0.05, 1e-2, 0.0, 1,
                z, z.copy(), z.copy(), z.copy(), f)
    prec = fsei.FSEI_FP64 if prec_name == "fp64" else fsei.FSEI_MIXED
    gpu, _ = pu.run_gpu(case, 2, prec)
    ref, _ = pu.run_oracle(case, 2)
    if prec_name == "fp64":
        _assert_fp64(gpu, ref)
    else:
        vel = np.sqrt(sum(np.linalg.norm(gpu[k] - ref[k]) ** 2 for k in "uvw")
                      / sum(np.linalg.norm(ref[k]) ** 2 for k in "uvw"))
        assert vel <= 1e-5, (vel, pu.compare(gpu, ref))


@pytest.mark.parametrize("nx", [64, 256])
@pytest.mark.parametrize("alpha", [0.02, 0.2, 0.45, 0.8])
@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
def test_x_line_carries_across_decay_lengths(fsei, nx, alpha, prec_name):
    """The register x solve sums the carries of the nearest D lanes where
    |alpha|^(4 D) is below the precision's tolerance (2^-32 single, 2^-62
    double) and D <= 8, and scans the whole cycle otherwise.  Re is set so
    that the x factor is alpha (beta/dx^2 = alpha / (1 - alpha)^2): in single
    precision D = 2, 4, 8 and the full scan, in double D = 3, 7 and the full
    scan twice; 64-wide rows put a line in 16 lanes of a warp, 256-wide ones
    across two warps.  Two steps from rest under a random force, against the
    oracle: 1e-12 per field in FP64, 1e-5 in velocity for mixed precision."""
    from paper_2103_15187_gb300.inputs import Case
    ny, nz, lx, dt = 8, 8, 2.0, 1e-2
    b = alpha / (1.0 - alpha) ** 2
    re = dt / (2.0 * b * (lx / nx) ** 2)
    rng = np.random.default_rng(nx + int(100 * alpha))
    z = np.zeros((nz, ny, nx))
    f = tuple(rng.standard_normal((nz, ny, nx)) for _ in range(3))
    f[2][0] = 0.0
    case = Case("carries", nx, ny, nz, lx, 1.0, Z_WALLS, 2.0, 1.5, re, dt, 0.0, 1,
                z, z.copy(), z.copy(), z.copy(), f)
    prec = fsei.FSEI_FP64 if prec_name == "fp64" else fsei.FSEI_MIXED
    gpu, _ = pu.run_gpu(case, 2, prec)
    ref, _ = pu.run_oracle(case, 2)
    if prec_name == "fp64":
        _assert_fp64(gpu, ref)
    else:
        vel = np.sqrt(sum(np.linalg.norm(gpu[k] - ref[k]) ** 2 for k in "uvw")
                      / sum(np.linalg.norm(ref[k]) ** 2 for k in "uvw"))
        assert vel <= 1e-5, (vel, pu.compare(gpu, ref))


@pytest.mark.parametrize("nx,ny,nz,walls", [(96, 24, 16, True), (48, 16, 12, False),
                                             (192, 12, 10, True), (384, 8, 8, True)])
@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
def test_rows_of_three_times_power_of_two(fsei, nx, ny, nz, walls, prec_name):
    """Rows of 3 x 2^m cells take 24-byte lanes in the row-resident RHS + x
    sweep (6 floats or 3 doubles per lane, nx / 6 or nx / 3 lanes, lines
    across up to four warps); body forces on the wall-bounded cases.  Three
    steps against the oracle: 1e-12 per field in FP64, 1e-5 in velocity for
    mixed precision; the schedule names the lane width."""
    if walls:
        case = inputs.case_channel(nx, ny, nz, steps=3, kmax=4.0, rms=0.3, seed=nx + nz,
                                   re=500.0, blobs=dict(nblobs=2, sigma=2.0, amp=3.0))
    else:
        case = inputs.case_periodic_random(nx, seed=nx, steps=3, re=400.0, ny=ny, nz=nz)
    prec = fsei.FSEI_FP64 if prec_name == "fp64" else fsei.FSEI_MIXED
    grid = pu.gpu_grid(case, prec)
    assert grid.schedule["rhs_cells_per_lane"] == (3 if prec_name == "fp64" else 6)
    gpu, _ = pu.run_gpu(case, 3, prec, grid=grid)
    ref, _ = pu.run_oracle(case, 3)
    if prec_name == "fp64":
        _assert_fp64(gpu, ref)
    else:
        vel = np.sqrt(sum(np.linalg.norm(gpu[k] - ref[k]) ** 2 for k in "uvw")
                      / sum(np.linalg.norm(ref[k]) ** 2 for k in "uvw"))
        assert vel <= 1e-5, (vel, pu.compare(gpu, ref))


def test_taylor_green_fp64_10_steps(fsei):
    """32^3 triply periodic Taylor-Green, Re 100, dt 1e-3, 10 steps."""
    case = inputs.case_taylor_green(32, steps=10)
    gpu, st = pu.run_gpu(case, 10, fsei.FSEI_FP64)
    ref, rst = pu.run_oracle(case, 10)
    _assert_fp64(gpu, ref)
    assert abs(st["kinetic_energy"] / rst[-1]["kinetic_energy"] - 1) < 1e-12
    assert st["max_div"] < 1e-12


@pytest.mark.parametrize("shape", [(48, 24, 36), (48, 36, 17)])
def test_channel_fp64_10_steps(fsei, shape):
    """Stretched channel with random solenoidal perturbation, Gaussian-blob
    body force, Poiseuille drive and CFL 0.5 time step; ragged extents."""
    nx, ny, nz = shape
    case = inputs.case_channel(nx, ny, nz, steps=10, kmax=4.0, rms=0.3, seed=nx,
                               blobs=dict(nblobs=3, sigma=3.0, amp=10.0))
    gpu, st = pu.run_gpu(case, 10, fsei.FSEI_FP64, per_call=4)
    ref, rst = pu.run_oracle(case, 10)
    _assert_fp64(gpu, ref)
    assert abs(st["dt_used"] / rst[-1]["dt_used"] - 1) < 1e-12
    assert abs(st["cfl"] / rst[-1]["cfl"] - 1) < 1e-12
    assert abs(st["kinetic_energy"] / rst[-1]["kinetic_energy"] - 1) < 1e-12


def test_periodic_random_fp64_10_steps(fsei):
    case = inputs.case_periodic_random(24, seed=3, steps=10)
    gpu, _ = pu.run_gpu(case, 10, fsei.FSEI_FP64)
    ref, _ = pu.run_oracle(case, 10)
    _assert_fp64(gpu, ref)


def test_mixed_channel_100_steps_against_fp64_oracle(fsei):
    """Mixed precision (FP32 fields, FP64 near-zero Poisson modes and
    reductions) stays within 1e-5 of the FP64 oracle in velocity after 100
    steps of a 64^3 stretched channel."""
    case = inputs.case_channel(64, 64, 64, steps=100, seed=2)
    gpu, _ = pu.run_gpu(case, 100, fsei.FSEI_MIXED)
    ref, _ = pu.run_oracle(case, 100)
    vel = _vel_err(gpu, ref)
    assert vel <= 1e-5, (vel, pu.compare(gpu, ref))


def _vel_err(gpu, ref):
    return np.sqrt(sum(np.linalg.norm(gpu[k] - ref[k]) ** 2 for k in "uvw")
                   / sum(np.linalg.norm(ref[k]) ** 2 for k in "uvw"))


def test_full_size_channel_fp64_10_steps(fsei):
    """256^3 stretched channel (the mixed-vs-FP64 workload: Re 2000, CFL 0.5,
    Poiseuille drive, RMS 0.1 perturbation) at full size: ten FP64 steps
    against ten oracle steps, 1e-12 per field, with the CFL time step, the
    CFL number and the kinetic energy of the last step."""
    case = inputs.case_channel(256, 256, 256, steps=10)
    gpu, st = pu.run_gpu(case, 10, fsei.FSEI_FP64)
    ref, rst = pu.run_oracle(case, 10)
    _assert_fp64(gpu, ref)
    assert st["max_div"] < 1e-9
    for key in ("dt_used", "cfl", "kinetic_energy"):
        assert abs(st[key] / rst[-1][key] - 1) < 1e-12, (key, st[key], rst[-1][key])


def test_mixed_channel_128_cubed_100_steps_against_fp64_oracle(fsei):
    """The mixed-precision gate against the FP64 oracle itself: 100 steps of
    the 128^3 version of the 256^3 channel (same Re, CFL, stretching and
    perturbation spectrum), velocity within 1e-5."""
    case = inputs.case_channel(128, 128, 128, steps=100, seed=2)
    gpu, st = pu.run_gpu(case, 100, fsei.FSEI_MIXED)
    ref, rst = pu.run_oracle(case, 100)
    err = _vel_err(gpu, ref)
    print("mixed vs oracle, 128^3 channel, 100 steps: velocity rel L2 %.3e" % err)
    assert err <= 1e-5, (err, pu.compare(gpu, ref))
    assert abs(st["dt_used"] / rst[-1]["dt_used"] - 1) < 1e-4


@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
def test_heart_scale_rows_and_y_transforms_against_oracle(fsei, prec_name):
    """The heart-scale box's x-y plane (512 x 512, its domain, Re, k^-5/3
    field and force blobs) on 16 stretched z cells: the RHS kernel's 512-wide
    rows (8 cells per lane in single precision) and the y transforms of
    length 512.  Three steps against the oracle: 1e-12 per field in FP64,
    1e-5 in velocity for mixed precision."""
    case = inputs.case_heart_scale(512, 512, 16, steps=3)
    prec = fsei.FSEI_FP64 if prec_name == "fp64" else fsei.FSEI_MIXED
    ref, _ = pu.run_oracle(case, 3)
    # every admissible width of the y transforms' tiles: 16 kx columns take
    # the second pass's pairs in two turns of 256 threads
    tried = []
    for cols in (None, 4, 8, 16):
        grid = pu.gpu_grid(case, prec)
        if prec_name == "mixed":
            assert grid.schedule["rhs_cells_per_lane"] == 8
        if cols is not None:
            try:
                grid.set_schedule({"ffty_columns_per_block": cols})
            except fsei.FseiError:
                continue
        tried.append(grid.schedule["ffty_columns_per_block"])
        gpu, st = pu.run_gpu(case, 3, prec, grid=grid)
        if prec_name == "fp64":
            _assert_fp64(gpu, ref)
        else:
            err = _vel_err(gpu, ref)
            assert err <= 1e-5, (cols, err, pu.compare(gpu, ref))
    assert 16 in tried, tried


def _poisson_768(fsei, prec_name, zbc):
    """The 768-cell z line of the heart-scale box under a 32 x 32 plane (its
    domain, stretched walls or a uniform periodic z): GPU Poisson solve and
    oracle on one seeded white-noise right-hand side."""
    import torch
    case = inputs.case_heart_scale(32, 32, 768, steps=3)
    prec = fsei.FSEI_FP64 if prec_name == "fp64" else fsei.FSEI_MIXED
    dtype = torch.float64 if prec_name == "fp64" else torch.float32
    stretch = case.stretch if zbc == Z_WALLS else 0.0
    grid = fsei.Grid(32, 32, 768, case.lx, case.ly, zbc=zbc, lz=2.0, stretch=stretch, prec=prec)
    if prec_name == "mixed":
        sched = grid.schedule
        assert (sched["poisson_lanes_per_line"], sched["poisson_rows_per_lane"]) == (32, 24)
    g = OGrid(32, 32, 768, case.lx, case.ly, zbc, lz=2.0, stretch=stretch)
    s = _compatible_rhs(g, 768)
    rhs = torch.tensor(s, dtype=dtype, device="cuda")
    phi = torch.empty_like(rhs)
    fsei.poisson_solve(grid, rhs, phi)
    torch.cuda.synchronize()
    # the oracle sees exactly the values the GPU was given
    ref = oracle_poisson(g, rhs.double().cpu().numpy())
    return phi.double().cpu().numpy(), ref


def test_heart_scale_z_line_poisson_fp64(fsei):
    """FP64 on the stretched 768-cell line (the chunked z solver).  Every
    Fourier mode but (0, 0) matches the oracle to 1e-12.  The (0, 0) mode is
    the pinned Neumann line itself: its condition number is about
    (2 / dz_min)^2 = 3e7 (dz_min = 3.8e-4 at the walls), and on this
    right-hand side, where that mode holds 95 % of the solution norm, the
    oracle's own FP64 solve already differs from an extended-precision one by
    2.4e-12.  The whole field is therefore held to 1e-11, four times that
    rounding floor."""
    gpu, ref = _poisson_768(fsei, "fp64", Z_WALLS)
    mg = gpu.mean(axis=(1, 2), keepdims=True)
    mr = ref.mean(axis=(1, 2), keepdims=True)
    assert pu.rel_l2(gpu - mg, ref - mr) <= FP64_TOL
    assert pu.rel_l2(gpu, ref) <= 1e-11


def _float_input_floor(g, s, tau=64.0):
    """Relative L2 error that representing the z systems in float alone
    causes: the Poisson solve of the oracle (double arithmetic) on the
    right-hand side, diagonals and off-diagonals of every z line rounded to
    float32, except the modes a mixed grid solves in double ((lambda_x +
    lambda_y) Lz^2 < tau, here with unrounded data).  A single-precision
    solver stores exactly these rounded values, so it cannot do better; for
    a low mode the diagonal (about 2 / (dz hc)) dwarfs the wavenumber
    lambda that separates the line's smallest eigenvalue from zero, and the
    rounding of the diagonal moves that eigenvalue by eps_32 (2 / (dz hc))
    / lambda relative."""
    nz, ny, nx = g.shape
    a, c, bz = z_poisson_coefficients(g)
    lam = (modified_wavenumbers(nx, g.dx)[None, :] + modified_wavenumbers(ny, g.dy)[:, None])
    sh = np.fft.fft2(s, axes=(1, 2))
    r32 = lambda x: x.astype(np.float32).astype(np.float64)  # noqa: E731
    b = r32(bz[:, None, None] - lam[None])
    d = r32(sh.real) + 1j * r32(sh.imag)
    b[:, 0, 0] = 1.0
    solve = thomas if g.walls else cyclic_thomas
    ph = solve(r32(a), b, r32(c), d, axis=0)
    exact = np.fft.fft2(oracle_poisson(g, s), axes=(1, 2))
    dbl = (lam * (g.zf[-1] - g.zf[0]) ** 2 < tau)
    ph[:, dbl] = exact[:, dbl]
    phi = np.real(np.fft.ifft2(ph, axes=(1, 2)))
    phi -= (phi * g.dz[:, None, None]).sum() / (g.dz.sum() * nx * ny)
    ref = oracle_poisson(g, s)
    return pu.rel_l2(phi, ref)


@pytest.mark.parametrize("zbc", [Z_WALLS, Z_PERIODIC])
def test_heart_scale_z_line_poisson_mixed(fsei, zbc):
    """Mixed precision on the 768-cell z line, white-noise right-hand side:
    the (0, 0) mode in double, the others in single precision through the
    heart-scale split of each mode line over 32 lanes of 24 rows (cyclic
    coupling for periodic z).  The error is held to ten times the floor that
    storing the z systems in float alone causes (_float_input_floor: 2.6e-5
    on the stretched walls, whose cells shrink to 3.8e-4; 1.6e-4 on the
    uniform periodic line, whose lowest float modes are nearly singular
    cyclic systems).  The step on this machine meets the 1e-5 velocity gate in
    the next test."""
    gpu, ref = _poisson_768(fsei, "mixed", zbc)
    case = inputs.case_heart_scale(32, 32, 768, steps=3)
    g = OGrid(32, 32, 768, case.lx, case.ly, zbc, lz=2.0,
              stretch=case.stretch if zbc == Z_WALLS else 0.0)
    s = _compatible_rhs(g, 768).astype(np.float32).astype(np.float64)
    floor = _float_input_floor(g, s)
    err = pu.rel_l2(gpu, ref)
    print("mixed Poisson, 32x32x768 zbc=%d, white noise: rel L2 %.3e (float-storage floor "
          "%.3e)" % (zbc, err, floor))
    assert err <= 10 * floor, (err, floor)


def test_heart_scale_z_line_poisson_periodic_fp64(fsei):
    """FP64 on a uniform periodic 768-cell line: 1e-12."""
    gpu, ref = _poisson_768(fsei, "fp64", Z_PERIODIC)
    err = pu.rel_l2(gpu, ref)
    assert err <= FP64_TOL, err


@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
def test_heart_scale_z_lines_three_steps(fsei, prec_name):
    """Three steps of the heart-scale box's 768-cell stretched z extent
    under a 32 x 32 plane (its domain, field and force blobs) against the
    oracle: 1e-12 per field in FP64, 1e-5 in velocity for mixed."""
    case = inputs.case_heart_scale(32, 32, 768, steps=3)
    prec = fsei.FSEI_FP64 if prec_name == "fp64" else fsei.FSEI_MIXED
    gpu, _ = pu.run_gpu(case, 3, prec)
    ref, _ = pu.run_oracle(case, 3)
    if prec_name == "fp64":
        _assert_fp64(gpu, ref)
    else:
        err = _vel_err(gpu, ref)
        print("mixed vs oracle, 32x32x768 heart-scale slice, 3 steps: %.3e" % err)
        assert err <= 1e-5, (err, pu.compare(gpu, ref))


def test_heart_scale_mixed_against_fp64_gpu(fsei):
    """512x512x768 heart-scale box (stretched walls, k^-5/3 field, 20 force
    blobs), the largest configuration, at full size: three mixed-precision
    steps against three FP64 steps of the GPU path (the kernel paths of this
    size meet the oracle in the two tests above, on slices of this box):
    velocity within 1e-5, divergence at round-off in both."""
    import torch
    case = inputs.case_heart_scale()
    out = {}
    for name, prec, dtype in (("fp64", fsei.FSEI_FP64, torch.float64),
                              ("mixed", fsei.FSEI_MIXED, torch.float32)):
        grid = pu.gpu_grid(case, prec)
        st = pu.to_device(pu.initial_state_np(case), dtype)
        f = pu.force_device(case, dtype)
        stats = fsei.step(grid, st, f, nsteps=3, **pu.params(case))
        assert stats["max_div"] < (1e-9 if name == "fp64" else 1e-2), stats
        out[name] = {k: st[k].double() for k in ("u", "v", "w")}
        del grid, st, f
        torch.cuda.empty_cache()
    num = sum(float(torch.linalg.vector_norm(out["mixed"][k] - out["fp64"][k]) ** 2) for k in "uvw")
    den = sum(float(torch.linalg.vector_norm(out["fp64"][k]) ** 2) for k in "uvw")
    assert (num / den) ** 0.5 <= 1e-5, (num / den) ** 0.5
