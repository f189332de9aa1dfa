"""Pins of the oracle's third-order Runge-Kutta variant of the fractional
step (Sec. 2.1 notes it beside Adams-Bashforth; the coefficients follow the
cited Rai & Moin / Verzicco & Orlandi low-storage scheme):

* linear regime: a Taylor-Green field of amplitude 1e-6 is a single Fourier
  mode that each sub-step multiplies by the factorised Crank-Nicolson factor
  of its sub-interval alpha_l dt, g_l = 1 - 2 beta_l Lambda /
  prod_d (1 + beta_l lambda_d) with beta_l = alpha_l dt / (2 Re): the mode
  after n steps is (g_1 g_2 g_3)^n (fixes the alpha_l and the sub-step
  structure);
* the advective part is third order in time: with Re -> infinity each
  sub-step is the low-storage RK3 update of du/dt = P H(u) (the projection
  removes the pressure gradient exactly), so the error at a fixed time falls
  by about 8 per halving of dt (fixes gamma_l and rho_l: any other weights
  of this form drop the order);
* a step keeps the velocity solenoidal and leaves a discrete Poiseuille
  profile steady."""

import numpy as np
import pytest

from oracle.grid import Grid, Z_PERIODIC, Z_WALLS
from oracle import step as st
from oracle.tridiag import thomas
from paper_2103_15187_gb300 import inputs


def _state(u, v, w, p=None):
    z = np.zeros_like(u)
    return {"u": u, "v": v, "w": w, "p": z.copy() if p is None else p,
            "hu": z.copy(), "hv": z.copy(), "hw": z.copy(), "have_prev_h": 0}


def _tg_coefficient(g, u):
    basis = np.sin(g.x_face())[None, None, :] * np.cos(g.y_centre())[None, :, None] \
        * np.cos(g.zc)[:, None, None]
    return (u * basis).sum() / (basis * basis).sum()


def test_rk3_coefficients_are_consistent():
    """alpha_l = gamma_l + rho_l sum to 1 (one full dt of the linear terms);
    rho_1 = 0 (a step needs no history)."""
    alpha = [a + b for a, b in zip(st.RK3_GAMMA, st.RK3_RHO)]
    assert abs(sum(alpha) - 1.0) < 1e-15
    assert st.RK3_RHO[0] == 0.0


def test_rk3_taylor_green_linear_regime_amplification():
    case = inputs.case_taylor_green(32, steps=10, amp=1e-6)
    g = Grid(32, 32, 32, case.lx, case.ly, Z_PERIODIC, lz=case.lz)
    re, dt, n = 100.0, 2e-2, 6
    s = _state(case.u, case.v, case.w)
    a0 = _tg_coefficient(g, s["u"])
    for _ in range(n):
        s, _stats = st.oracle_step_rk3(g, s, None, re=re, dt=dt)
    lam = (2 - 2 * np.cos(g.dx)) / g.dx ** 2
    gfull = 1.0
    for a_l in (8 / 15, 2 / 15, 1 / 3):
        beta = a_l * dt / (2 * re)
        gfull *= 1 - 2 * beta * 3 * lam / (1 + beta * lam) ** 3
    ratio = _tg_coefficient(g, s["u"]) / a0
    assert abs(ratio / gfull ** n - 1) <= 1e-10


def test_rk3_advection_third_order_in_time():
    """Inviscid (Re = 1e30) random solenoidal field on a 16^3 periodic box,
    t = 0.3: errors against a 256-step solution for 6, 12 and 24 steps fall
    with observed order >= 2.8 in every component."""
    case = inputs.case_periodic_random(16, seed=12, steps=1)
    g = Grid(16, 16, 16, case.lx, case.ly, Z_PERIODIC, lz=case.lz)

    def run(nsteps):
        s = _state(case.u, case.v, case.w)
        for _ in range(nsteps):
            s, _st = st.oracle_step_rk3(g, s, None, re=1e30, dt=0.3 / nsteps)
        return s

    ref = run(256)
    errs = []
    for n in (6, 12, 24):
        s = run(n)
        errs.append([np.abs(s[k] - ref[k]).max() for k in "uvw"])
    errs = np.array(errs)
    orders = np.log2(errs[:-1] / errs[1:])
    assert np.all(orders >= 2.8), (errs, orders)


@pytest.mark.parametrize("zbc", [Z_WALLS, Z_PERIODIC])
def test_rk3_step_is_solenoidal(zbc):
    g = Grid(24, 20, 18, 2 * np.pi, np.pi, zbc, lz=2.0, stretch=2.0)
    rng = np.random.default_rng(14)
    u, v, w = (rng.standard_normal(g.shape) for _ in range(3))
    if g.walls:
        w[0] = 0.0
    f = tuple(rng.standard_normal(g.shape) for _ in range(3))
    s = _state(u, v, w)
    for _ in range(2):
        s, stats = st.oracle_step_rk3(g, s, f, re=500.0, dt=2e-3)
        hmin = min(g.dx, g.dy, g.dz.min())
        scale = max(np.abs(s[k]).max() for k in "uvw") / hmin
        assert stats["max_div"] <= 1e-13 * scale
        if g.walls:
            assert np.all(s["w"][0] == 0.0)


def test_rk3_discrete_poiseuille_is_steady():
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
    for _ in range(30):
        s, _stats = st.oracle_step_rk3(g, s, None, re=re, cfl=1.0, fconst=(fx, 0.0, 0.0))
    assert np.max(np.abs(s["u"] - u0)) <= 1e-12 * np.max(np.abs(u0))
    assert np.max(np.abs(s["v"])) <= 1e-13 and np.max(np.abs(s["w"])) <= 1e-13
