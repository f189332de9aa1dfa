"""Pins of the oracle's Carreau-Yasuda stress (Sec. 2.1): for a constant
excess viscosity the stress divergence is c (L u + G D u) with the
Newtonian operators (the discrete form of div(2E) = lap u + grad div u);
the Newtonian limits give no correction; a shear flow u = U(z) reduces to
a 1-D formula written out here from the mesh; the stress divergence obeys
the discrete energy identity sum(u . div tau) = -sum(tau : grad u); the law
has its zero-shear value 1 and its power-law slope n - 1 at high shear; a
step with the law keeps the velocity solenoidal and reduces to the
Newtonian step when n = 1."""

import numpy as np
import pytest

from oracle.grid import Grid, Z_PERIODIC, Z_WALLS
from oracle import operators as op
from oracle import rheology as rh
from oracle import step as st

CY = dict(lam=3.0, n=0.35, a=2.0, eta_inf=0.06)


def _fields(g, seed):
    rng = np.random.default_rng(seed)
    u, v, w = (rng.standard_normal(g.shape) for _ in range(3))
    if g.walls:
        w[0] = 0.0
    return u, v, w


@pytest.mark.parametrize("zbc", [Z_WALLS, Z_PERIODIC])
def test_constant_viscosity_is_laplacian_plus_grad_div(zbc):
    g = Grid(12, 10, 14, 2.0, 1.5, zbc, lz=1.7, stretch=1.6)
    u, v, w = _fields(g, 1)
    c = 0.37
    nu = np.full(g.shape, c)
    hx, hy, hz = rh.stress_divergence(g, u, v, w, nu, *rh.excess_viscosity_edges(g, nu))
    lu, lv, lw = op.viscous(g, u, v, w)
    gx, gy, gz = op.gradient(g, op.divergence(g, u, v, w))
    for h, l, gr in ((hx, lu, gx), (hy, lv, gy), (hz, lw, gz)):
        ref = c * (l + gr)
        if g.walls:
            ref[0] = 0.0 if h is hz else ref[0]
        assert np.max(np.abs(h - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("params", [dict(CY, n=1.0), dict(CY, eta_inf=1.0)])
def test_newtonian_limits_give_no_correction(params):
    g = Grid(12, 10, 14, 2.0, 1.5, Z_WALLS, stretch=1.6)
    u, v, w = _fields(g, 2)
    for h in rh.non_newtonian_term(g, u, v, w, 100.0, **params):
        assert np.max(np.abs(h)) == 0.0


def test_shear_flow_reduces_to_one_dimensional_formula():
    nz, re = 20, 40.0
    g = Grid(8, 6, nz, 1.0, 1.0, Z_WALLS, stretch=1.7)
    zf = np.array([np.tanh(1.7 * (2.0 * k / nz - 1.0)) / np.tanh(1.7) for k in range(nz + 1)])
    zc = 0.5 * (zf[1:] + zf[:-1])
    dz = zf[1:] - zf[:-1]
    hc = np.concatenate([[zc[0] - zf[0]], zc[1:] - zc[:-1], [zf[-1] - zc[-1]]])
    U = np.sin(2.0 * zc) + 0.3 * zc ** 2
    u = U[:, None, None] * np.ones(g.shape)
    z = np.zeros(g.shape)
    hx, hy, hz = rh.non_newtonian_term(g, u, z, z.copy(), re, **CY)
    Ue = np.concatenate([[0.0], U, [0.0]])            # wall values
    e = (Ue[1:] - Ue[:-1]) / hc                       # du/dz at faces 0..nz
    gdot = np.abs(e[:-1] + e[1:]) / 2.0               # 2 |E_xz| averaged to centres
    lam, n, a, ei = CY["lam"], CY["n"], CY["a"], CY["eta_inf"]
    nu = (ei + (1 - ei) * (1 + (lam * gdot) ** a) ** ((n - 1) / a) - 1.0) / re
    nu_e = np.concatenate([[nu[0]], 0.5 * (nu[1:] + nu[:-1]), [nu[-1]]])
    tau = nu_e * e
    want = (tau[1:] - tau[:-1]) / dz
    assert np.max(np.abs(hx - want[:, None, None])) <= 1e-13 * np.max(np.abs(want))
    assert np.max(np.abs(hy)) < 1e-15 and np.max(np.abs(hz)) < 1e-15


def test_stress_divergence_energy_identity():
    """Periodic uniform box, arbitrary viscosities at centres and edges:
    sum(u hx + v hy + w hz) = -sum(2 nu_c (Exx^2 + Eyy^2 + Ezz^2))
    - sum(4 (nu_xy Exy^2 + nu_xz Exz^2 + nu_yz Eyz^2)) (equal volumes)."""
    g = Grid(10, 12, 8, 1.3, 1.1, Z_PERIODIC, lz=0.9)
    u, v, w = _fields(g, 3)
    rng = np.random.default_rng(4)
    nu_c, nu_xy = rng.uniform(0.1, 1.0, g.shape), rng.uniform(0.1, 1.0, g.shape)
    nz = g.nz
    nu_xz = np.empty((nz + 1,) + g.shape[1:])
    nu_yz = np.empty((nz + 1,) + g.shape[1:])
    nu_xz[:nz] = rng.uniform(0.1, 1.0, g.shape)
    nu_yz[:nz] = rng.uniform(0.1, 1.0, g.shape)
    nu_xz[nz], nu_yz[nz] = nu_xz[0], nu_yz[0]
    hx, hy, hz = rh.stress_divergence(g, u, v, w, nu_c, nu_xy, nu_xz, nu_yz)
    (exx, eyy, ezz), exy, exz, eyz = rh.strain_rates(g, u, v, w)
    lhs = (u * hx + v * hy + w * hz).sum()
    rhs = -(2 * nu_c * (exx ** 2 + eyy ** 2 + ezz ** 2)).sum() - 4 * (
        (nu_xy * exy ** 2).sum() + (nu_xz[:nz] * exz[:nz] ** 2).sum()
        + (nu_yz[:nz] * eyz[:nz] ** 2).sum())
    assert abs(lhs / rhs - 1) < 1e-12


def test_carreau_yasuda_limits():
    assert rh.carreau_yasuda(0.0, **CY) == 1.0
    g1, g2 = 1e6, 2e6
    e1 = rh.carreau_yasuda(g1, **CY) - CY["eta_inf"]
    e2 = rh.carreau_yasuda(g2, **CY) - CY["eta_inf"]
    assert abs(np.log(e2 / e1) / np.log(2.0) - (CY["n"] - 1.0)) < 1e-6
    assert rh.carreau_yasuda(1e30, **CY) == pytest.approx(CY["eta_inf"], abs=1e-8)


def test_step_with_rheology():
    """Stretched channel: divergence at round-off with the law on; with
    n = 1 the step is the Newtonian step bit for bit."""
    g = Grid(16, 12, 18, 2.0, 1.0, Z_WALLS, stretch=1.5)
    u, v, w = _fields(g, 5)
    z = np.zeros(g.shape)
    s0 = {"u": u, "v": v, "w": w, "p": z, "hu": z, "hv": z, "hw": z, "have_prev_h": 0}
    s, stats = st.oracle_step(g, s0, None, re=30.0, dt=2e-3, rheology=CY)
    hmin = min(g.dx, g.dy, g.dz.min())
    assert stats["max_div"] <= 1e-13 * max(np.abs(s[k]).max() for k in "uvw") / hmin
    a, _ = st.oracle_step(g, s0, None, re=30.0, dt=2e-3, rheology=dict(CY, n=1.0))
    b, _ = st.oracle_step(g, s0, None, re=30.0, dt=2e-3)
    for k in ("u", "v", "w", "p", "hu"):
        assert np.array_equal(a[k], b[k])


@pytest.mark.parametrize("case", ["v(x)", "u(y)", "w(x)", "w(y)"])
def test_periodic_shear_flows_reduce_to_one_dimensional_formula(case):
    """A velocity component varying along one periodic direction only (all
    else 0) on a periodic box: one shear component, the difference e_i of
    neighbouring values over the spacing at edge i, gdot = |e_i + e_{i+1}| / 2
    at the centres between them, nu' at edge i the mean of its two cells, and
    the term (nu'_{i+1} e_{i+1} - nu'_i e_i) / h at the moving component's
    points.  Catches an average taken over the wrong neighbours."""
    n, re = 16, 25.0
    g = Grid(n, n, n, 1.0, 1.0, Z_PERIODIC, lz=1.0)
    h = 1.0 / n
    s = np.arange(n) * h
    F = np.sin(2 * np.pi * s) + 0.4 * np.cos(6 * np.pi * s)    # at the moving points
    comp, axis = {"v(x)": (1, 2), "u(y)": (0, 1), "w(x)": (2, 2), "w(y)": (2, 1)}[case]
    shape = [1, 1, 1]
    shape[axis] = n
    fld = [np.zeros(g.shape) for _ in range(3)]
    fld[comp] = F.reshape(shape) * np.ones(g.shape)
    terms = rh.non_newtonian_term(g, *fld, re, **CY)
    # the moving component's points sit at centres along `axis` when the
    # component differs from the axis direction; the edges then sit at the
    # faces i h, between centres i - 1 and i
    e = (F - np.roll(F, 1)) / h                     # at edge i
    gdot = np.abs(e + np.roll(e, -1)) / 2.0         # at the centre between edges i, i + 1
    lam, nn, a, ei = CY["lam"], CY["n"], CY["a"], CY["eta_inf"]
    nu = (ei + (1 - ei) * (1 + (lam * gdot) ** a) ** ((nn - 1) / a) - 1.0) / re
    nu_e = 0.5 * (nu + np.roll(nu, 1))              # edge i between centres i - 1, i
    tau = nu_e * e
    want = (np.roll(tau, -1) - tau) / h             # at the centre i
    got = terms[comp]
    assert np.max(np.abs(got - want.reshape(shape))) <= 1e-12 * np.max(np.abs(want))
    for c in range(3):
        if c != comp:
            assert np.max(np.abs(terms[c])) < 1e-13
