"""Pins of the oracle's staggered operators (Sec. 2.1: central second-order
differences on a staggered mesh) against properties the mathematics fixes:
summation by parts between D and G, D G equal to the compound Laplacian,
Fourier-mode eigenvalues of the periodic second difference, self-adjointness
of the stretched-z viscous operators in the volume-weighted inner product,
second-order consistency of the advection operator with -div(uu), axis
symmetry of the three advection components, and conservation of kinetic
energy by the advection operator for a discretely solenoidal field."""

import numpy as np
import pytest
import sympy as sp

from oracle.grid import Grid, Z_PERIODIC, Z_WALLS
from oracle import operators as op
from paper_2103_15187_gb300 import inputs


def _grids():
    return [
        Grid(8, 6, 7, 2.0, 1.5, Z_WALLS, stretch=2.0),
        Grid(6, 8, 5, 1.0, 3.0, Z_WALLS, stretch=0.0),
        Grid(6, 5, 8, 2.0, 1.0, Z_PERIODIC, lz=1.7),
    ]


def _rand(g, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal(g.shape) for _ in range(4)]


@pytest.mark.parametrize("g", _grids())
def test_summation_by_parts(g):
    """sum_c phi (D u) dV_c = -sum_f (G phi).u dV_f  (G = -D^T)."""
    u, v, w, phi = _rand(g, 1)
    w = op.wall_w(g, w)
    lhs = (phi * op.divergence(g, u, v, w) * g.cell_volume_uvp()).sum()
    gx, gy, gz = op.gradient(g, phi)
    rhs = -((gx * u + gy * v) * g.cell_volume_uvp()).sum() \
        - (gz * w * g.cell_volume_w()).sum()
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs) + 1.0)


@pytest.mark.parametrize("g", _grids())
def test_compound_laplacian_is_div_grad(g):
    phi = _rand(g, 2)[0]
    lap = op.laplacian_p(g, phi)
    dg = op.divergence(g, *op.gradient(g, phi))
    assert np.max(np.abs(lap - dg)) <= 1e-12 * np.max(np.abs(lap))


@pytest.mark.parametrize("g", _grids())
def test_viscous_operators_self_adjoint(g):
    """L_z = W^-1 S with S symmetric: <a, L b>_W = <L a, b>_W with
    W = dz_k at z-centres and W = hc_k at z-faces."""
    a, b, c, d = _rand(g, 3)
    vol_c = g.cell_volume_uvp()
    l1 = (a * op.lapz_centre(g, b) * vol_c).sum()
    l2 = (op.lapz_centre(g, a) * b * vol_c).sum()
    assert abs(l1 - l2) <= 1e-12 * (abs(l1) + 1.0)
    c, d = op.wall_w(g, c), op.wall_w(g, d)
    vol_w = g.cell_volume_w()
    l3 = (c * op.lapz_face(g, d) * vol_w).sum()
    l4 = (op.lapz_face(g, c) * d * vol_w).sum()
    assert abs(l3 - l4) <= 1e-12 * (abs(l3) + 1.0)
    # Poisson operator: symmetric and negative semi-definite, constants in
    # its null space
    l5 = (a * op.laplacian_p(g, b) * vol_c).sum()
    l6 = (op.laplacian_p(g, a) * b * vol_c).sum()
    assert abs(l5 - l6) <= 1e-12 * (abs(l5) + 1.0)
    assert (a * op.laplacian_p(g, a) * vol_c).sum() < 0
    assert np.max(np.abs(op.laplacian_p(g, np.ones(g.shape)))) < 1e-9


def test_periodic_second_difference_eigenvalues():
    """lap_xy e^{i(kx x + ky y)} = -(lambda_x + lambda_y) e^{...} with
    lambda = (2 - 2 cos(k h)) / h^2 (modified wavenumber)."""
    g = Grid(16, 12, 4, 2 * np.pi, 3.0, Z_PERIODIC, lz=1.0)
    kx, ky = 3, 2
    x = g.x_centre()[None, None, :]
    y = g.y_centre()[None, :, None]
    ax = 2 * np.pi * kx / g.lx
    ay = 2 * np.pi * ky / g.ly
    mode = np.exp(1j * (ax * x + ay * y)) * np.ones((g.nz, 1, 1))
    lam = (2 - 2 * np.cos(ax * g.dx)) / g.dx ** 2 \
        + (2 - 2 * np.cos(ay * g.dy)) / g.dy ** 2
    out = op.lap_xy(g, mode)
    assert np.max(np.abs(out + lam * mode)) < 1e-12 * lam


def _analytic_fields():
    X, Y, Z = sp.symbols("x y z")
    uu = sp.sin(X) * sp.cos(Y) * sp.sin(Z) + sp.Rational(3, 10) * sp.cos(2 * X)
    vv = sp.cos(X + Y) * sp.cos(Z) + sp.Rational(1, 5) * sp.sin(Y)
    ww = sp.sin(X) * sp.sin(Y + Z) + sp.Rational(1, 4) * sp.cos(Z)
    hu = -(sp.diff(uu * uu, X) + sp.diff(vv * uu, Y) + sp.diff(ww * uu, Z))
    hv = -(sp.diff(uu * vv, X) + sp.diff(vv * vv, Y) + sp.diff(ww * vv, Z))
    hw = -(sp.diff(uu * ww, X) + sp.diff(vv * ww, Y) + sp.diff(ww * ww, Z))
    f = lambda e: sp.lambdify((X, Y, Z), e, "numpy")  # noqa: E731
    return [f(e) for e in (uu, vv, ww, hu, hv, hw)]


def _sample(fun, g, sx, sy, sz):
    """fun at staggered points: s* = 0 face, 1 centre."""
    x = g.x_centre() if sx else g.x_face()
    y = g.y_centre() if sy else g.y_face()
    z = g.zc if sz else g.zf[:-1]
    return np.broadcast_to(fun(x[None, None, :], y[None, :, None],
                               z[:, None, None]), g.shape).astype(float)


def test_advection_second_order_consistency():
    """H -> -div(uu) at second order on a uniform triply periodic grid
    (catches a wrong average, sign or index in any of the nine fluxes)."""
    fu, fv, fw, fhu, fhv, fhw = _analytic_fields()
    errs = []
    for n in (16, 32, 64):
        g = Grid(n, n, n, 2 * np.pi, 2 * np.pi, Z_PERIODIC, lz=2 * np.pi)
        u = _sample(fu, g, 0, 1, 1)
        v = _sample(fv, g, 1, 0, 1)
        w = _sample(fw, g, 1, 1, 0)
        hu, hv, hw = op.advection(g, u, v, w)
        e = max(np.max(np.abs(hu - _sample(fhu, g, 0, 1, 1))),
                np.max(np.abs(hv - _sample(fhv, g, 1, 0, 1))),
                np.max(np.abs(hw - _sample(fhw, g, 1, 1, 0))))
        errs.append(e)
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.9), (errs, orders)


def test_advection_axis_symmetry():
    """Exchanging the x and z axes of a periodic cube maps u <-> w; the
    advection operator must map H_u <-> H_w and H_v -> H_v accordingly."""
    n = 8
    g = Grid(n, n, n, 2 * np.pi, 2 * np.pi, Z_PERIODIC, lz=2 * np.pi)
    u, v, w, _ = _rand(g, 4)
    hu, hv, hw = op.advection(g, u, v, w)
    t = lambda a: np.ascontiguousarray(a.transpose(2, 1, 0))  # noqa: E731
    hu2, hv2, hw2 = op.advection(g, t(w), t(v), t(u))
    assert np.max(np.abs(hu2 - t(hw))) < 1e-12
    assert np.max(np.abs(hv2 - t(hv))) < 1e-12
    assert np.max(np.abs(hw2 - t(hu))) < 1e-12
    # x <-> y exchange
    s = lambda a: np.ascontiguousarray(a.transpose(0, 2, 1))  # noqa: E731
    hu3, hv3, hw3 = op.advection(g, s(v), s(u), s(w))
    assert np.max(np.abs(hu3 - s(hv))) < 1e-12
    assert np.max(np.abs(hv3 - s(hu))) < 1e-12
    assert np.max(np.abs(hw3 - s(hw))) < 1e-12


@pytest.mark.parametrize("zbc", [Z_PERIODIC, Z_WALLS])
def test_advection_conserves_kinetic_energy(zbc):
    """sum u.H dV = 0 for a discretely solenoidal field on a uniform mesh (the
    divergence form with two-point averages is energy-conserving when the
    discrete continuity equation holds)."""
    nx, ny, nz = 16, 12, 10
    lz = 2.0
    g = Grid(nx, ny, nz, 2 * np.pi, 3.0, zbc, lz=lz, stretch=0.0)
    rng = np.random.Generator(np.random.PCG64(11))
    zf = inputs.z_faces(nz, zbc, lz, 0.0)
    u, v, w = inputs.solenoidal_field(rng, nx, ny, nz, g.lx, g.ly, zf, zbc,
                                      1.0, 4.0, 0.0, mmax=3)
    assert np.max(np.abs(op.divergence(g, u, v, w))) < 1e-12
    hu, hv, hw = op.advection(g, u, v, w)
    e = ((u * hu + v * hv) * g.cell_volume_uvp()).sum() \
        + (w * hw * g.cell_volume_w()).sum()
    scale = (np.abs(u * hu) * g.cell_volume_uvp()).sum()
    assert abs(e) <= 1e-13 * scale
