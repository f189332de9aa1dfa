"""Pins of the oracle's immersed-boundary operators (Sec. 2.1 Eq. 4 and
Eqs. 5-7, Sec. 3.2): moving-least-squares transfer operators with the
linear basis reproduce linear fields exactly and sum to one; the fit is the
weighted least-squares line of numpy's lstsq (weights written out here from
the node coordinates); spreading conserves the total force and is the
volume-weighted transpose of the interpolation; the direct forcing of a
linear field is known in closed form; face loads of linear pressure and
velocity fields are exact; nodal loads split every face load in thirds; a
uniform pressure on a closed surface gives no net load."""

import numpy as np
import pytest

from oracle.grid import Grid, Z_PERIODIC, Z_WALLS
from oracle import ib
from paper_2103_15187_gb300 import inputs


def _channel():
    return Grid(24, 20, 28, 2.0, 1.6, Z_WALLS, stretch=1.8)


def _tanh_faces(nz, s):
    return np.array([np.tanh(s * (2.0 * k / nz - 1.0)) / np.tanh(s) for k in range(nz + 1)])


def _node_coords(g, loc, k, j, i):
    """Coordinates of node (k, j, i) of a staggered component, written out
    from the mesh definition (faces x_i = i dx, centres (i + 1/2) dx; z
    faces from the tanh law, centres their midpoints)."""
    zf = _tanh_faces(g.nz, 1.8) if g.walls else np.arange(g.nz + 1) * (g.zf[-1] / g.nz)
    x = i * g.dx if loc == ib.U else (i + 0.5) * g.dx
    y = j * g.dy if loc == ib.V else (j + 0.5) * g.dy
    z = zf[k] if loc == ib.W else 0.5 * (zf[k] + zf[k + 1])
    return np.array([x, y, z])


POINTS = [np.array([0.77, 0.53, 0.11]), np.array([1.31, 0.92, -0.43]),
          np.array([0.05, 1.55, 0.6])]      # the last one's support wraps in x and y


@pytest.mark.parametrize("loc", [ib.U, ib.V, ib.W, ib.P])
@pytest.mark.parametrize("pt", range(3))
def test_transfer_operators_reproduce_linear_fields(loc, pt):
    g = _channel()
    xb = POINTS[pt]
    idx, phi = ib.transfer(g, loc, xb)
    assert len(idx) == 27
    assert abs(phi.sum() - 1.0) < 1e-13
    rel = []
    for (k, j, i) in idx:
        d = _node_coords(g, loc, k, j, i) - xb
        d[0] = (d[0] + 0.5 * g.lx) % g.lx - 0.5 * g.lx
        d[1] = (d[1] + 0.5 * g.ly) % g.ly - 0.5 * g.ly
        rel.append(d)
    rel = np.array(rel)
    assert np.max(np.abs(phi @ rel)) < 1e-13


def test_fit_is_weighted_least_squares():
    """The fit of an arbitrary field equals numpy's least-squares solution
    of sqrt(w_k) [1, s_k] a = sqrt(w_k) f_k with w_k = exp(-|s_k|^2), s_k
    the node offsets over the nearest node's control extents."""
    g = _channel()
    rng = np.random.default_rng(3)
    field = rng.standard_normal(g.shape)
    xb = POINTS[1]
    for loc in (ib.U, ib.W):
        idx, _, _ = ib.support(g, loc, xb)
        kc = idx[13][0]                     # centre node of the support
        zf = _tanh_faces(g.nz, 1.8)
        hz = (0.5 * (zf[kc + 1] - zf[kc - 1]) if loc == ib.W else zf[kc + 1] - zf[kc])
        h = np.array([g.dx, g.dy, hz])
        s = np.array([_node_coords(g, loc, k, j, i) - xb for (k, j, i) in idx]) / h
        w = np.exp(-(s * s).sum(axis=1))
        M = np.sqrt(w)[:, None] * np.hstack([np.ones((27, 1)), s])
        rhs = np.sqrt(w) * np.array([field[k] for k in idx])
        a, *_ = np.linalg.lstsq(M, rhs, rcond=None)
        val, grad = ib.fit(g, field, loc, xb)
        assert abs(val - a[0]) < 1e-12 * max(1.0, abs(a[0]))
        assert np.max(np.abs(grad - a[1:] / h)) < 1e-10 * np.max(np.abs(a[1:] / h))


def test_fit_exact_for_linear_fields_value_and_gradient():
    g = _channel()
    c0, G = 0.3, np.array([1.7, -0.4, 2.2])
    for loc in (ib.U, ib.V, ib.W, ib.P):
        f = np.zeros(g.shape)
        for k in range(g.nz):
            for j in range(g.ny):
                for i in range(g.nx):
                    f[k, j, i] = c0 + G @ _node_coords(g, loc, k, j, i)
        x = POINTS[1]
        val, grad = ib.fit(g, f, loc, x)
        assert abs(val - (c0 + G @ x)) < 1e-12
        assert np.max(np.abs(grad - G)) < 1e-11


def _markers(g, n, seed):
    rng = np.random.default_rng(seed)
    xb = np.column_stack([rng.uniform(0, g.lx, n), rng.uniform(0, g.ly, n),
                          rng.uniform(-0.7, 0.7, n)])
    ub = rng.standard_normal((n, 3))
    dvb = rng.uniform(0.5, 2.0, n) * g.dx * g.dy * 0.05
    return xb, ub, dvb


def test_spreading_conserves_force_and_is_interpolation_transpose():
    g = _channel()
    rng = np.random.default_rng(5)
    u, v, w = (rng.standard_normal(g.shape) for _ in range(3))
    w[0] = 0.0
    xb, ub, dvb = _markers(g, 25, 6)
    dt = 3e-3
    (fx, fy, fz), ui = ib.ib_forcing(g, u, v, w, xb, ub, dvb, dt)
    F = (ub - ui) / dt
    for c, f in enumerate((fx, fy, fz)):
        vol = ib.node_volumes(g, c)
        assert abs((f * vol).sum() / (F[:, c] * dvb).sum() - 1) < 1e-12
    # <I u, G>_markers = <u, S G>_nodes for marker values G: spreading G
    # through the forcing path (u = 0, U_b = G dt) against interpolation
    Gm = rng.standard_normal((25, 3))
    z = np.zeros(g.shape)
    (sx, sy, sz), _ = ib.ib_forcing(g, z, z, z, xb, Gm * dt, dvb, dt)
    for c, (fld, s) in enumerate(zip((u, v, w), (sx, sy, sz))):
        lhs = (ui[:, c] * Gm[:, c] * dvb).sum()
        rhs = (fld * s * ib.node_volumes(g, c)).sum()
        assert abs(lhs / rhs - 1) < 1e-12


def test_direct_forcing_of_a_linear_field():
    """u = G . x at every component's points: the interpolated velocity is
    exact, so F_b = (U_b - G . x_b) / dt."""
    g = Grid(16, 16, 16, 1.0, 1.0, Z_PERIODIC, lz=1.0)
    G = np.array([[0.5, -0.2, 0.1], [0.3, 0.4, -0.6], [-0.1, 0.2, 0.7]])
    f = []
    for c in range(3):
        a = np.zeros(g.shape)
        for k in range(g.nz):
            for j in range(g.ny):
                for i in range(g.nx):
                    a[k, j, i] = G[c] @ _node_coords(g, c, k, j, i)
        f.append(a)
    xb = np.array([[0.41, 0.52, 0.47], [0.61, 0.33, 0.58]])   # supports inside, no wrap
    ub = np.array([[1.0, 0.0, -1.0], [0.5, 0.5, 0.5]])
    _, ui = ib.ib_forcing(g, f[0], f[1], f[2], xb, ub, np.ones(2), 0.1)
    assert np.max(np.abs(ui - xb @ G.T)) < 1e-12


def test_face_loads_of_linear_fields():
    """p = p0 + Gp . x and u_i = M_ij x_j (M traceless): at every probe the
    fits are exact, so a one-sided face carries (-(p0 + Gp . (x_f + h n)) n
    + Re^-1 (M + M^T) n) A and a two-sided one -(2 h Gp . n) n A (the stress
    is the same on both sides)."""
    g = Grid(32, 32, 32, 2.0, 2.0, Z_PERIODIC, lz=2.0)
    p0, Gp = 0.7, np.array([0.3, -1.1, 0.6])
    M = np.array([[0.4, 0.9, -0.3], [0.2, -0.1, 0.5], [-0.7, 0.6, -0.3]])
    re, h = 50.0, 0.07
    def fill(loc, fn):
        a = np.zeros(g.shape)
        for k in range(g.nz):
            for j in range(g.ny):
                for i in range(g.nx):
                    a[k, j, i] = fn(_node_coords(g, loc, k, j, i))
        return a
    p = fill(ib.P, lambda x: p0 + Gp @ x)
    u, v, w = (fill(c, lambda x, c=c: M[c] @ x) for c in range(3))
    surf = inputs.ib_surface((1.0, 1.0, 1.0), 0.3, 1)
    xf, nf, af = surf["xf"], surf["nf"], surf["af"]
    for two in (False, True):
        ts = np.full(len(xf), two)
        F, _ = ib.face_loads(g, p, u, v, w, xf, nf, af, ts, h, re)
        for f in range(len(xf)):
            n = nf[f]
            if two:
                want = -(2 * h * (Gp @ n)) * n * af[f]
            else:
                want = (-(p0 + Gp @ (xf[f] + h * n)) * n + (M + M.T) @ n / re) * af[f]
            assert np.max(np.abs(F[f] - want)) < 1e-11


def test_nodal_loads_and_closed_surface():
    surf = inputs.ib_surface((0.0, 0.0, 0.0), 1.0, 2)
    rng = np.random.default_rng(9)
    F = rng.standard_normal((len(surf["tris"]), 3))
    Fn = ib.nodal_loads(F, surf["tris"], len(surf["verts"]))
    assert np.max(np.abs(Fn.sum(axis=0) - F.sum(axis=0))) < 1e-12
    one = ib.nodal_loads(F[:1], surf["tris"][:1], len(surf["verts"]))
    for n in surf["tris"][0]:
        assert np.max(np.abs(one[n] - F[0] / 3)) < 1e-15
    # a uniform pressure pushes a closed surface nowhere: sum n_f A_f = 0
    Fp = -2.5 * surf["nf"] * surf["af"][:, None]
    assert np.max(np.abs(Fp.sum(axis=0))) < 1e-13


def test_support_tie_goes_to_the_node_whose_volume_holds_the_point():
    """A point exactly on the x face i dx is halfway between centres i - 1
    and i: it lies in cell i, so the centre support is centred on i; exactly
    on the centre (i + 1/2) dx it is halfway between faces i and i + 1 and
    lies in the control volume [(i + 1/2) dx, (i + 3/2) dx) of face i + 1."""
    g = Grid(16, 16, 16, 1.0, 1.0, Z_PERIODIC, lz=1.0)
    x = np.array([5 / 16, 0.43, 0.51])
    idx, _, _ = ib.support(g, ib.V, x)      # v: x at the centres
    assert idx[13][2] == 5
    x = np.array([5.5 / 16, 0.43, 0.51])
    idx, _, _ = ib.support(g, ib.U, x)      # u: x at the faces
    assert idx[13][2] == 6
