"""Pins of the oracle's pressure-increment Poisson solve (Sec. 2.1, the elliptic
equation of the fractional-step method): a dense LU solve of the assembled
compound operator D G with one row replaced by the gauge constraint (small
grids), a single Fourier mode reduced to one tridiagonal system, and the
residual at a larger size."""

import numpy as np
import pytest

from oracle.grid import Grid, Z_PERIODIC, Z_WALLS
from oracle import operators as op
from oracle.poisson import oracle_poisson


def _compatible_rhs(g, seed):
    rng = np.random.default_rng(seed)
    s = rng.standard_normal(g.shape)
    vol = g.cell_volume_uvp()
    return s - (s * vol).sum() / (vol.sum() * g.nx * g.ny)


def _dense_dg(g):
    """Assemble D G column by column from the divergence and gradient
    operators (each pinned separately)."""
    n = g.nx * g.ny * g.nz
    m = np.empty((n, n))
    e = np.zeros(n)
    for col in range(n):
        e[:] = 0.0
        e[col] = 1.0
        m[:, col] = op.divergence(g, *op.gradient(g, e.reshape(g.shape))).ravel()
    return m


GRIDS = [
    Grid(4, 4, 4, 1.0, 1.0, Z_WALLS, stretch=2.0),
    Grid(8, 6, 5, 2.0, 1.0, Z_WALLS, stretch=1.5),
    Grid(6, 8, 8, 2 * np.pi, np.pi, Z_WALLS, stretch=2.0),
    Grid(6, 4, 6, 1.0, 2.0, Z_PERIODIC, lz=3.0),
    Grid(8, 8, 8, 2 * np.pi, 2 * np.pi, Z_PERIODIC, lz=2 * np.pi),
]


@pytest.mark.parametrize("g", GRIDS)
def test_poisson_matches_dense_lu(g):
    s = _compatible_rhs(g, 5)
    m = _dense_dg(g)
    vol = np.broadcast_to(g.cell_volume_uvp(), g.shape).ravel()
    # replace one (redundant) row by the gauge: volume-weighted mean zero
    m[0, :] = vol
    rhs = s.ravel().copy()
    rhs[0] = 0.0
    ref = np.linalg.solve(m, rhs).reshape(g.shape)
    phi = oracle_poisson(g, s)
    err = np.linalg.norm(phi - ref) / np.linalg.norm(ref)
    assert err <= 1e-12, err


def test_single_mode_reduces_to_one_tridiagonal():
    """s = e^{i(kx x + ky y)} q(z): phi = e^{...} r(z) with
    (L_z - lambda) r = q, one dense 1-D solve."""
    g = Grid(16, 12, 10, 2.0, 3.0, Z_WALLS, stretch=2.0)
    kx, ky = 3, 5
    rng = np.random.default_rng(9)
    q = rng.standard_normal(g.nz)
    ex = np.exp(2j * np.pi * kx * np.arange(g.nx) / g.nx)
    ey = np.exp(2j * np.pi * ky * np.arange(g.ny) / g.ny)
    modal = ey[:, None] * ex[None, :]
    s = q[:, None, None] * modal[None]
    phi_re = oracle_poisson(g, s.real)
    phi_im = oracle_poisson(g, s.imag)
    phi = phi_re + 1j * phi_im
    lam = (2 - 2 * np.cos(2 * np.pi * kx / g.nx)) / g.dx ** 2 \
        + (2 - 2 * np.cos(2 * np.pi * ky / g.ny)) / g.dy ** 2
    lz = np.empty((g.nz, g.nz))
    for k in range(g.nz):
        e = np.zeros((g.nz, 1, 1))
        e[k] = 1.0
        lz[:, k] = op.lapz_poisson(g, e)[:, 0, 0]
    r = np.linalg.solve(lz - lam * np.eye(g.nz), q)
    ref = r[:, None, None] * modal[None]
    assert np.max(np.abs(phi - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("zbc", [Z_WALLS, Z_PERIODIC])
def test_residual_and_gauge_at_larger_size(zbc):
    g = Grid(48, 40, 36, 2 * np.pi, np.pi, zbc, lz=2.0, stretch=2.0)
    s = _compatible_rhs(g, 6)
    phi = oracle_poisson(g, s)
    res = op.laplacian_p(g, phi) - s
    assert np.max(np.abs(res)) <= 1e-11 * np.max(np.abs(s))
    mean = (phi * g.cell_volume_uvp()).sum()
    assert abs(mean) <= 1e-12 * np.abs(phi * g.cell_volume_uvp()).sum()


def _naive_dft(n):
    """The O(n^2) DFT matrix, forward sign e^{-i}, unnormalised."""
    j = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(j, j) / n)


@pytest.mark.parametrize("n", [32, 64, 96, 128])
def test_fft_step_against_naive_dft(n):
    """The transform the oracle's Poisson solve applies (numpy's FFT, a
    library step) against the naive O(n^2) DFT: forward e^{-i} unnormalised,
    inverse with 1/n; and that DFT diagonalises the periodic second
    difference with the oracle's modified wavenumbers, -lambda_m."""
    from oracle.poisson import modified_wavenumbers
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    F = _naive_dft(n)
    ref = F @ x
    assert np.linalg.norm(np.fft.fft(x) - ref) <= 1e-13 * np.linalg.norm(ref)
    assert np.linalg.norm(np.fft.ifft(ref) - x) <= 1e-13 * np.linalg.norm(x)
    h = 2 * np.pi / n
    d2 = (np.roll(np.eye(n), 1, axis=1) + np.roll(np.eye(n), -1, axis=1) - 2 * np.eye(n)) / h ** 2
    lam = modified_wavenumbers(n, h)
    diag = F @ d2 @ np.linalg.inv(F)
    assert np.max(np.abs(diag - np.diag(-lam))) <= 1e-10 * lam.max()


def test_fft2_axes_are_y_and_x():
    """The oracle's two-dimensional transform runs along y and x of a
    [nz][ny][nx] field (axes 1 and 2), not along z."""
    rng = np.random.default_rng(7)
    s = rng.standard_normal((3, 6, 8))
    ref = np.einsum("ab,kbc,dc->kad", _naive_dft(6), s, _naive_dft(8))
    assert np.max(np.abs(np.fft.fft2(s, axes=(1, 2)) - ref)) <= 1e-12
