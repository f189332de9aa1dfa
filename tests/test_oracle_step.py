"""Pins of the oracle's fractional step (Sec. 2.1, Eq. 3 with gamma = 3/2,
rho = -1/2; Sec. 3.1 approximate factorisation with Thomas / Sherman-Morrison
sweeps): sweep residuals against the viscous operator, the closed-form
single-mode amplification of the factorised Crank-Nicolson step, discrete
divergence after projection, Taylor-Green decay (linear regime exactly, full
amplitude against exp(-3t/Re)), a discrete Poiseuille steady state, and
second-order convergence on a manufactured solution."""

import numpy as np
import pytest
import sympy as sp

from oracle.grid import Grid, Z_PERIODIC, Z_WALLS
from oracle import operators as op
from oracle import step as st
from oracle.tridiag import thomas
from paper_2103_15187_gb300 import inputs


def _state(u, v, w, p=None):
    z = np.zeros_like(u)
    return {"u": u, "v": v, "w": w, "p": z.copy() if p is None else p,
            "hu": z.copy(), "hv": z.copy(), "hw": z.copy(), "have_prev_h": 0}


@pytest.mark.parametrize("zbc", [Z_WALLS, Z_PERIODIC])
def test_sweeps_invert_one_dimensional_operators(zbc):
    """(I - beta L_d) applied to the sweep output returns its input, with L_d
    the operator pieces the explicit right-hand side uses."""
    g = Grid(12, 10, 9, 2.0, 1.0, zbc, lz=1.5, stretch=2.0)
    rng = np.random.default_rng(3)
    d = rng.standard_normal(g.shape)
    beta = 0.37e-2
    q = st.sweep_x(g, beta, d)
    lx = (op.xp(q) - 2 * q + op.xm(q)) / g.dx ** 2
    assert np.max(np.abs(q - beta * lx - d)) < 1e-13
    q = st.sweep_y(g, beta, d)
    ly = (op.yp(q) - 2 * q + op.ym(q)) / g.dy ** 2
    assert np.max(np.abs(q - beta * ly - d)) < 1e-13
    q = st.sweep_z_centre(g, beta, d)
    assert np.max(np.abs(q - beta * op.lapz_centre(g, q) - d)) < 1e-12
    dw = op.wall_w(g, d)
    q = st.sweep_z_face(g, beta, dw)
    res = q - beta * op.lapz_face(g, q) - dw
    assert np.max(np.abs(res)) < 1e-12


def test_factorised_crank_nicolson_single_mode():
    """For a Fourier mode on a uniform periodic box the factorised solve is
    multiplication by 1 / prod_d (1 + beta lambda_d)."""
    g = Grid(16, 12, 10, 2.0, 3.0, Z_PERIODIC, lz=1.5)
    k = (3, 2, 4)
    beta = 0.05
    x = g.x_face()[None, None, :]
    y = g.y_centre()[None, :, None]
    z = g.zc[:, None, None]
    ang = [2 * np.pi * k[0] / g.lx, 2 * np.pi * k[1] / g.ly,
           2 * np.pi * k[2] / 1.5]
    mode = np.cos(ang[0] * x + ang[1] * y + ang[2] * z) * np.ones(g.shape)
    lam = [(2 - 2 * np.cos(a * h)) / h ** 2
           for a, h in zip(ang, (g.dx, g.dy, g.dz[0]))]
    out = st.sweep_z_centre(g, beta, st.sweep_y(g, beta,
                                                 st.sweep_x(g, beta, mode)))
    fac = 1.0 / np.prod([1 + beta * l for l in lam])
    assert np.max(np.abs(out - fac * mode)) <= 1e-14 * 4


def _tg_coefficient(g, u):
    basis = np.sin(g.x_face())[None, None, :] * np.cos(g.y_centre())[None, :, None] \
        * np.cos(g.zc)[:, None, None]
    return (u * basis).sum() / (basis * basis).sum()


def test_taylor_green_linear_regime_amplification():
    """Amplitude 1e-6, 32^3, 10 steps: the (1,1,1) coefficient is g^n with
    g = 1 - 2 beta sum(lambda) / prod(1 + beta lambda); advection is
    O(1e-12) and does not feed this mode."""
    case = inputs.case_taylor_green(32, steps=10, amp=1e-6)
    g = Grid(32, 32, 32, case.lx, case.ly, Z_PERIODIC, lz=case.lz)
    s = _state(case.u, case.v, case.w)
    a0 = _tg_coefficient(g, s["u"])
    for _ in range(10):
        s, _stats = st.oracle_step(g, s, None, re=case.re, dt=case.dt)
    beta = case.dt / (2 * case.re)
    lam = (2 - 2 * np.cos(g.dx)) / g.dx ** 2
    gfac = 1 - 2 * beta * 3 * lam / (1 + beta * lam) ** 3
    ratio = _tg_coefficient(g, s["u"]) / a0
    assert abs(ratio / gfac ** 10 - 1) <= 1e-10
    assert abs(_tg_coefficient(g, -s["v"].transpose(0, 2, 1)) / a0
               / gfac ** 10 - 1) <= 1e-10


def test_taylor_green_full_amplitude():
    """32^3, Re = 100, dt = 1e-3, 10 steps: the (1,1,1) coefficient follows
    exp(-3 t / Re) (nonlinear transfer to it is second order in t), kinetic
    energy decays monotonically, divergence stays at round-off."""
    case = inputs.case_taylor_green(32, steps=10)
    g = Grid(32, 32, 32, case.lx, case.ly, Z_PERIODIC, lz=case.lz)
    s = _state(case.u, case.v, case.w)
    a0 = _tg_coefficient(g, s["u"])
    ke_prev = np.inf
    for n in range(10):
        s, stats = st.oracle_step(g, s, None, re=case.re, dt=case.dt)
        assert stats["kinetic_energy"] < ke_prev
        ke_prev = stats["kinetic_energy"]
        assert stats["max_div"] <= 1e-12
    t = 10 * case.dt
    assert abs(_tg_coefficient(g, s["u"]) / a0 - np.exp(-3 * t / case.re)) <= 1e-4


@pytest.mark.parametrize("zbc", [Z_WALLS, Z_PERIODIC])
def test_projection_leaves_divergence_at_round_off(zbc):
    g = Grid(24, 20, 18, 2 * np.pi, np.pi, zbc, lz=2.0, stretch=2.0)
    rng = np.random.default_rng(4)
    u, v, w = (rng.standard_normal(g.shape) for _ in range(3))
    f = tuple(rng.standard_normal(g.shape) for _ in range(3))
    s = _state(u, v, op.wall_w(g, w))
    for _ in range(3):
        s, stats = st.oracle_step(g, s, f, re=500.0, dt=2e-3)
        hmin = min(g.dx, g.dy, g.dz.min())
        scale = max(np.abs(s["u"]).max(), np.abs(s["v"]).max(),
                    np.abs(s["w"]).max()) / hmin
        assert stats["max_div"] <= 1e-13 * scale
        if g.walls:
            assert np.all(s["w"][0] == 0.0)


def test_discrete_poiseuille_is_steady():
    """u solving Re^-1 L_z u = -f_x discretely (one Dirichlet tridiagonal
    solve) with v = w = 0 stays steady for 100 steps."""
    re = 2000.0
    g = Grid(16, 8, 32, 2 * np.pi, np.pi, Z_WALLS, stretch=2.0)
    fx = 2.0 / re
    lo = 1.0 / (g.hc[:-1] * g.dz)
    hi = 1.0 / (g.hc[1:] * g.dz)
    prof = thomas(lo, -(lo + hi), hi, np.full(g.nz, -fx * re))
    u = prof[:, None, None] * np.ones(g.shape)
    z = np.zeros(g.shape)
    s = _state(u, z.copy(), z.copy())
    u0 = u.copy()
    for _ in range(100):
        s, _stats = st.oracle_step(g, s, None, re=re, cfl=0.5,
                                   fconst=(fx, 0.0, 0.0))
    assert np.max(np.abs(s["u"] - u0)) <= 1e-12 * np.max(np.abs(u0))
    assert np.max(np.abs(s["v"])) <= 1e-13 and np.max(np.abs(s["w"])) <= 1e-13
    # and the profile is within O(h^2) of the continuous 1 - z^2
    assert np.max(np.abs(prof - (1 - g.zc ** 2))) < 1e-2


# ------------------------------------------------- manufactured solution ----
def _mms():
    X, Y, Z, T, RE = sp.symbols("x y z t re")
    gz = (1 - Z ** 2) ** 2
    tt = sp.exp(-T)
    a1, a2, a3 = sp.Rational(1), sp.Rational(1, 2), sp.Rational(-3, 4)
    ax = gz * tt * a1 * sp.sin(X) * sp.cos(Y)
    ay = gz * tt * a2 * sp.cos(X) * sp.sin(Y)
    az = gz * tt * a3 * sp.sin(X) * sp.sin(Y)
    u = sp.diff(az, Y) - sp.diff(ay, Z)
    v = sp.diff(ax, Z) - sp.diff(az, X)
    w = sp.diff(ay, X) - sp.diff(ax, Y)
    p = tt * sp.cos(X) * sp.cos(Y) * sp.sin(sp.pi * Z / 2)
    vel = (u, v, w)
    f = []
    for c, uc in enumerate(vel):
        conv = sum(sp.diff(vel[d] * uc, s) for d, s in enumerate((X, Y, Z)))
        lap = sum(sp.diff(uc, s, 2) for s in (X, Y, Z))
        f.append(sp.diff(uc, T) + conv + sp.diff(p, (X, Y, Z)[c]) - lap / RE)
    lam = lambda e: sp.lambdify((X, Y, Z, T, RE), e, "numpy")  # noqa: E731
    return [lam(e) for e in (u, v, w, p)], [lam(e) for e in f]


def _at(fun, g, loc, t, re):
    sx, sy, sz = loc
    x = g.x_centre() if sx else g.x_face()
    y = g.y_centre() if sy else g.y_face()
    z = g.zc if sz else g.zf[:-1]
    return np.broadcast_to(fun(x[None, None, :], y[None, :, None],
                               z[:, None, None], t, re),
                           g.shape).astype(float).copy()


LOC = ((0, 1, 1), (1, 0, 1), (1, 1, 0), (1, 1, 1))


@pytest.mark.slow
def test_manufactured_solution_second_order():
    """u_e = curl(g(z) T(t) a(x, y)), g = (1 - z^2)^2 (no-slip, solenoidal),
    p_e = T cos x cos y sin(pi z / 2), T = e^-t, f from the PDE evaluated at
    t^{n+1/2}; stretched walls, dt proportional to h: observed order >= 1.9
    in u, v, w and p (p modulo its mean).  The pressure of the Crank-Nicolson
    step is the Lagrange multiplier of a step centred at t^{n+1/2}, so it is
    compared with p_e at t_end - dt/2 (against p_e(t_end) it is only first
    order, an O(dt) time shift)."""
    (fu, fv, fw, fp), ff = _mms()
    re = 10.0
    t_end = 0.2
    errs = []
    for n in (16, 32, 64):
        g = Grid(n, n, 3 * n // 2, 2 * np.pi, 2 * np.pi, Z_WALLS, stretch=1.5)
        nsteps = {16: 8, 32: 16, 64: 32}[n]
        dt = t_end / nsteps
        s = _state(*(_at(fn, g, LOC[c], 0.0, re) for c, fn in
                     enumerate((fu, fv, fw))), p=_at(fp, g, LOC[3], 0.0, re))
        s["w"][0] = 0.0
        for it in range(nsteps):
            th = (it + 0.5) * dt
            f = tuple(_at(ff[c], g, LOC[c], th, re) for c in range(3))
            s, _st = st.oracle_step(g, s, f, re=re, dt=dt)
        e = []
        for c, (name, fn) in enumerate(zip("uvwp", (fu, fv, fw, fp))):
            t_cmp = t_end - 0.5 * dt if name == "p" else t_end
            ex = _at(fn, g, LOC[c], t_cmp, re)
            num = s[name]
            if name == "p":
                vol = g.cell_volume_uvp()
                num = num - (num * vol).sum() / (vol.sum() * n * n)
                ex = ex - (ex * vol).sum() / (vol.sum() * n * n)
            e.append(np.max(np.abs(num - ex)))
        errs.append(e)
    errs = np.array(errs)
    orders = np.log2(errs[:-1] / errs[1:])
    assert np.all(orders[-1] >= 1.9), (errs, orders)


# ------------------------------------------------ CFL time step and energy --
def _tanh_faces(nz, s):
    """Stretched wall faces written out from the tanh clustering law, apart
    from the oracle's grid module."""
    return np.array([np.tanh(s * (2.0 * k / nz - 1.0)) / np.tanh(s)
                     for k in range(nz + 1)])


def test_cfl_dt_uniform_flow_periodic_box():
    """A uniform stream u = U on a periodic box: every cell sees |U|/dx, so
    dt = CFL dx / |U| exactly."""
    g = Grid(12, 10, 8, 3.0, 2.0, Z_PERIODIC, lz=1.6)
    U = -1.7
    u = np.full(g.shape, U)
    z = np.zeros(g.shape)
    dt = st.oracle_cfl_dt(g, u, z, z.copy(), 0.5)
    assert abs(dt - 0.5 * (3.0 / 12) / abs(U)) <= 1e-15


def test_cfl_dt_single_cell_sum_on_stretched_channel():
    """One u face, one v face and one interior w face that all bound cell
    (k0, j0, i0) of a stretched channel carry U, V, W; every other value is 0.
    The centre speeds are two-face averages, so that cell's speed is
    |U|/(2 dx) + |V|/(2 dy) + |W|/(2 dz_k0), larger than that of any of its
    neighbours (each sees one of the three halves), and
    dt = CFL / that sum.  Reading face values instead of averages doubles it;
    weighting the w term by hc_k instead of dz_k changes it; dropping a
    component lowers it."""
    nx, ny, nz = 10, 8, 12
    g = Grid(nx, ny, nz, 2.0, 1.5, Z_WALLS, stretch=2.0)
    zf = _tanh_faces(nz, 2.0)
    dz = zf[1:] - zf[:-1]
    k0, j0, i0 = 5, 3, 4
    U, V, W = 0.9, -1.3, 0.7
    u = np.zeros(g.shape)
    v = np.zeros(g.shape)
    w = np.zeros(g.shape)
    u[k0, j0, i0] = U          # x face i0 = the low-x face of cell i0
    v[k0, j0, i0] = V          # y face j0 = the low-y face of cell j0
    w[k0, j0, i0] = W          # z face k0 = the low-z face of cell k0
    spd = abs(U) / (2 * 2.0 / nx) + abs(V) / (2 * 1.5 / ny) + abs(W) / (2 * dz[k0])
    # the neighbours each see one half-term only
    assert spd > max(abs(U) / (2 * 2.0 / nx), abs(V) / (2 * 1.5 / ny),
                     abs(W) / (2 * min(dz[k0 - 1], dz[k0])))
    dt = st.oracle_cfl_dt(g, u, v, w, 0.5)
    assert abs(dt / (0.5 / spd) - 1) <= 1e-14


def test_cfl_dt_w_only_asymmetric_faces():
    """w on the stretched channel only, on two neighbouring interior faces k1
    and k1+1 with unequal values A and B: the centre between them has
    w_c = (A+B)/2, its neighbours A/2 and B/2; dt = CFL / max over those
    three of |w_c| / dz_k, computed here from the tanh faces directly."""
    nx, ny, nz = 8, 6, 16
    g = Grid(nx, ny, nz, 1.0, 1.0, Z_WALLS, stretch=2.0)
    zf = _tanh_faces(nz, 2.0)
    dz = zf[1:] - zf[:-1]
    k1 = 2                      # near the bottom wall: dz varies fast there
    A, B = 1.0, -0.25
    w = np.zeros(g.shape)
    w[k1, 2, 3] = A
    w[k1 + 1, 2, 3] = B
    z = np.zeros(g.shape)
    cand = [abs(A) / 2 / dz[k1 - 1], abs(A + B) / 2 / dz[k1], abs(B) / 2 / dz[k1 + 1]]
    dt = st.oracle_cfl_dt(g, z, z.copy(), w, 0.8)
    assert abs(dt / (0.8 / max(cand)) - 1) <= 1e-14
    # the bottom wall face is not an unknown: a value stored there is ignored
    w2 = w.copy()
    w2[0, 1, 1] = 50.0
    assert st.oracle_cfl_dt(g, z, z.copy(), w2, 0.8) == dt


@pytest.mark.parametrize("comp", ["u", "v", "w"])
def test_kinetic_energy_closed_form_walls(comp):
    """Constant component C on a stretched channel, the others 0.  u and v
    live at the centres (weights dx dy dz_k, summing to lx ly 2), so
    KE = lx ly C^2.  w lives on the interior faces k = 1..nz-1 (weights
    dx dy hc_k, which sum to the distance between the first and last centres,
    2 - dz_0/2 - dz_{nz-1}/2); the bottom wall face is not counted even when
    a value is stored there."""
    nx, ny, nz = 6, 4, 10
    lx, ly = 1.5, 0.75
    g = Grid(nx, ny, nz, lx, ly, Z_WALLS, stretch=2.0)
    zf = _tanh_faces(nz, 2.0)
    dz = zf[1:] - zf[:-1]
    C = 0.6
    f = {k: np.zeros(g.shape) for k in "uvw"}
    f[comp][...] = C
    ke = st.oracle_stats(g, f["u"], f["v"], f["w"], 1e-3)["kinetic_energy"]
    if comp == "w":
        want = 0.5 * lx * ly * C * C * (2.0 - dz[0] / 2 - dz[-1] / 2)
    else:
        want = 0.5 * lx * ly * C * C * 2.0
    assert abs(ke / want - 1) <= 1e-14


def test_kinetic_energy_closed_form_periodic_modes():
    """Periodic box: u = a cos(2 pi x / lx) at the u points, v = b sin(2 pi y
    / ly) at the v points, w = c cos(2 pi z / lz) at the w faces.  Each
    squared mode sums to half its point count, so sum(u^2 dV) = a^2 lx ly lz
    / 2 and KE = (a^2 + b^2 + c^2) lx ly lz / 4."""
    g = Grid(8, 12, 10, 2.0, 3.0, Z_PERIODIC, lz=1.25)
    a, b, c = 0.5, -1.5, 2.0
    x = np.arange(8) * (2.0 / 8)
    y = np.arange(12) * (3.0 / 12)
    zfw = np.arange(10) * (1.25 / 10)
    u = a * np.cos(2 * np.pi * x / 2.0)[None, None, :] * np.ones(g.shape)
    v = b * np.sin(2 * np.pi * y / 3.0)[None, :, None] * np.ones(g.shape)
    w = c * np.cos(2 * np.pi * zfw / 1.25)[:, None, None] * np.ones(g.shape)
    ke = st.oracle_stats(g, u, v, w, 1e-3)["kinetic_energy"]
    assert abs(ke / ((a * a + b * b + c * c) * 2.0 * 3.0 * 1.25 / 4) - 1) <= 1e-14
