"""One fractional step of the AB2 / Crank-Nicolson integrator (Sec. 2.1, Eq. 3
with gamma = 3/2, rho = -1/2; fractional-step method; Sec. 3.1 approximate
factorisation into one tridiagonal system per direction).  Test
infrastructure only (see package header).

Reading of the sub-steps (the paper defers them to its citations of Kim &
Moin and Verzicco & Orlandi), with beta = dt / (2 Re):

1. dt: given, or from the CFL number, dt = CFL / max over cells of
   |u_c|/dx + |v_c|/dy + |w_c|/dz_k (u_c, v_c, w_c: two-face averages at the
   cell centre), recomputed from u^n every step.
2. gamma, rho = 3/2, -1/2; on the first step (no H^{n-1}) gamma, rho = 1, 0.
3. RHS = dt [gamma H^n + rho H^{n-1} + Re^-1 L u^n - G p^n + f]  (Eq. 3 in
   delta form with the predictor pressure p^n).
4. du = (I - beta L_z)^-1 (I - beta L_y)^-1 (I - beta L_x)^-1 RHS;
   u* = u^n + du.  x and y systems are cyclic (Sherman-Morrison).
5. phi = (D G)^-1 (D u* / dt) with the gauge of ``poisson``.
6. u^{n+1} = u* - dt G phi;  p^{n+1} = p^n + phi - beta (D G) phi.
   H^n becomes the stored history.

f is the body force the caller passes for the step (the immersed-boundary
forcing enters the fractional step as a given field), plus an optional
uniform part ``fconst``.
"""

import numpy as np

from . import operators as op
from .poisson import oracle_poisson
from .rheology import non_newtonian_term
from .tridiag import thomas, cyclic_thomas


def _centre_speeds(g, u, v, w):
    w = op.wall_w(g, w)
    uc = 0.5 * (u + op.xp(u))
    vc = 0.5 * (v + op.yp(v))
    wc = 0.5 * (w + op.zup(w, g))
    return (np.abs(uc) / g.dx + np.abs(vc) / g.dy
            + np.abs(wc) / g.dz[:, None, None])


def oracle_cfl_dt(g, u, v, w, cfl):
    """dt = CFL / max_cells(|u_c|/dx + |v_c|/dy + |w_c|/dz_k)."""
    return cfl / _centre_speeds(g, u, v, w).max()


def oracle_stats(g, u, v, w, dt):
    """Per-step statistics of the new state: CFL number with the step's dt,
    max |D u|, kinetic energy 1/2 sum(u^2 dV)."""
    ke = 0.5 * ((u * u * g.cell_volume_uvp()).sum()
                + (v * v * g.cell_volume_uvp()).sum()
                + (w * w * g.cell_volume_w()).sum())
    return {
        "cfl": dt * _centre_speeds(g, u, v, w).max(),
        "max_div": np.abs(op.divergence(g, u, v, w)).max(),
        "kinetic_energy": ke,
    }


# ------------------------------------------------ implicit viscous sweeps ---
def sweep_x(g, beta, d):
    r = beta / g.dx ** 2
    n = g.nx
    return cyclic_thomas(np.full(n, -r), np.full(n, 1 + 2 * r),
                         np.full(n, -r), d, axis=2)


def sweep_y(g, beta, d):
    r = beta / g.dy ** 2
    n = g.ny
    return cyclic_thomas(np.full(n, -r), np.full(n, 1 + 2 * r),
                         np.full(n, -r), d, axis=1)


def z_centre_coefficients(g, beta):
    """(I - beta L_z) at z-centre points (u, v): Dirichlet walls."""
    lo = beta / (g.hc[:-1] * g.dz)
    hi = beta / (g.hc[1:] * g.dz)
    return -lo, 1.0 + lo + hi, -hi


def z_face_coefficients(g, beta):
    """(I - beta L_z) at w faces k = 0..nz-1 (with walls row 0 is unused)."""
    nz = g.nz
    dz_below = np.roll(g.dz, 1)          # dz_{k-1}
    lo = beta / (dz_below * g.hc[:nz])
    hi = beta / (g.dz * g.hc[:nz])
    return -lo, 1.0 + lo + hi, -hi


def sweep_z_centre(g, beta, d):
    a, b, c = z_centre_coefficients(g, beta)
    if g.walls:
        return thomas(a, b, c, d, axis=0)
    return cyclic_thomas(a, b, c, d, axis=0)


def sweep_z_face(g, beta, d):
    a, b, c = z_face_coefficients(g, beta)
    if g.walls:
        out = np.zeros_like(d)
        out[1:] = thomas(a[1:], b[1:], c[1:], d[1:], axis=0)
        return out
    return cyclic_thomas(a, b, c, d, axis=0)


# ----------------------------------------------------------------- step ----
def oracle_step(g, state, f=None, re=100.0, dt=1e-3, cfl=0.0, gamma=1.5,
                rho=-0.5, fconst=(0.0, 0.0, 0.0), rheology=None):
    """One step n -> n+1.  `state` is a dict with float64 arrays u, v, w, p,
    hu, hv, hw (H^{n-1}) and the flag have_prev_h; `f` is None or a tuple
    (fx, fy, fz).  rheology: None (Newtonian) or a dict lam, n, a, eta_inf of
    the Carreau-Yasuda law, whose explicit remainder joins H (see
    rheology.py).  Returns (new_state, stats)."""
    u, v, w, p = state["u"], state["v"], state["w"], state["p"]
    w = op.wall_w(g, w)
    if cfl > 0.0:
        dt = oracle_cfl_dt(g, u, v, w, cfl)
    if not state.get("have_prev_h", 0):
        gamma, rho = 1.0, 0.0
    beta = dt / (2.0 * re)

    hu, hv, hw = op.advection(g, u, v, w)
    if rheology is not None:
        nu_u, nu_v, nu_w = non_newtonian_term(g, u, v, w, re, **rheology)
        hu, hv, hw = hu + nu_u, hv + nu_v, hw + nu_w
    lu, lv, lw = op.viscous(g, u, v, w)
    gx, gy, gz = op.gradient(g, p)
    if f is None:
        fx = fy = fz = 0.0
    else:
        fx, fy, fz = f
    rhs_u = dt * (gamma * hu + rho * state["hu"] + lu / re - gx + fx
                  + fconst[0])
    rhs_v = dt * (gamma * hv + rho * state["hv"] + lv / re - gy + fy
                  + fconst[1])
    rhs_w = dt * (gamma * hw + rho * state["hw"] + lw / re - gz + fz
                  + fconst[2])
    if g.walls:
        rhs_w[0] = 0.0

    du = sweep_z_centre(g, beta, sweep_y(g, beta, sweep_x(g, beta, rhs_u)))
    dv = sweep_z_centre(g, beta, sweep_y(g, beta, sweep_x(g, beta, rhs_v)))
    dw = sweep_z_face(g, beta, sweep_y(g, beta, sweep_x(g, beta, rhs_w)))
    us, vs, ws = u + du, v + dv, w + dw
    if g.walls:
        ws[0] = 0.0

    phi = oracle_poisson(g, op.divergence(g, us, vs, ws) / dt)
    px, py, pz = op.gradient(g, phi)
    un, vn, wn = us - dt * px, vs - dt * py, ws - dt * pz
    pn = p + phi - beta * op.laplacian_p(g, phi)

    new = {"u": un, "v": vn, "w": wn, "p": pn, "hu": hu, "hv": hv,
           "hw": hw, "have_prev_h": 1}
    stats = {"dt_used": dt}
    stats.update(oracle_stats(g, un, vn, wn, dt))
    return new, stats


def oracle_run(g, state, nsteps, f=None, **params):
    """nsteps successive steps; returns (state, list of stats)."""
    all_stats = []
    for _ in range(nsteps):
        state, st = oracle_step(g, state, f, **params)
        all_stats.append(st)
    return state, all_stats


# -------------------------------------------------- RK3 variant (Sec. 2.1) --
# The paper notes that a third-order Runge-Kutta scheme is implemented beside
# Adams-Bashforth without writing it out; its solver follows the cited Rai &
# Moin and Verzicco & Orlandi, whose low-storage scheme takes three
# sub-steps l = 1, 2, 3 with
#     gamma_l = 8/15, 5/12, 3/4,   rho_l = 0, -17/60, -5/12,
#     alpha_l = gamma_l + rho_l = 8/15, 2/15, 1/3  (sum 1),
# the advection weighted by gamma_l (this sub-step) and rho_l (the previous
# one), the viscous, pressure and force terms by alpha_l (Crank-Nicolson
# over the sub-interval alpha_l dt).
RK3_GAMMA = (8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0)
RK3_RHO = (0.0, -17.0 / 60.0, -5.0 / 12.0)


def rk3_substep(g, u, v, w, p, h_prev, dt, gamma_l, rho_l, alpha_l, re, f, fconst):
    """One sub-step of the RK3 / Crank-Nicolson fractional step:
    RHS = dt [gamma_l H^l + rho_l H^{l-1}] + alpha_l dt [Re^-1 L u^l - G p^l
    + f]; (I - beta_l L_z)(I - beta_l L_y)(I - beta_l L_x) du = RHS with
    beta_l = alpha_l dt / (2 Re); u* = u^l + du; phi = (D G)^-1 D u* /
    (alpha_l dt); u^{l+1} = u* - alpha_l dt G phi; p^{l+1} = p^l + phi -
    beta_l D G phi.  Returns (u, v, w, p, H^l)."""
    w = op.wall_w(g, w)
    hu, hv, hw = op.advection(g, u, v, w)
    lu, lv, lw = op.viscous(g, u, v, w)
    gx, gy, gz = op.gradient(g, p)
    fx, fy, fz = (0.0, 0.0, 0.0) if f is None else f
    adt = alpha_l * dt
    beta = adt / (2.0 * re)
    rhs_u = dt * (gamma_l * hu + rho_l * h_prev[0]) + adt * (lu / re - gx + fx + fconst[0])
    rhs_v = dt * (gamma_l * hv + rho_l * h_prev[1]) + adt * (lv / re - gy + fy + fconst[1])
    rhs_w = dt * (gamma_l * hw + rho_l * h_prev[2]) + adt * (lw / re - gz + fz + fconst[2])
    if g.walls:
        rhs_w[0] = 0.0
    du = sweep_z_centre(g, beta, sweep_y(g, beta, sweep_x(g, beta, rhs_u)))
    dv = sweep_z_centre(g, beta, sweep_y(g, beta, sweep_x(g, beta, rhs_v)))
    dw = sweep_z_face(g, beta, sweep_y(g, beta, sweep_x(g, beta, rhs_w)))
    us, vs, ws = u + du, v + dv, w + dw
    if g.walls:
        ws[0] = 0.0
    phi = oracle_poisson(g, op.divergence(g, us, vs, ws) / adt)
    px, py, pz = op.gradient(g, phi)
    return (us - adt * px, vs - adt * py, ws - adt * pz,
            p + phi - beta * op.laplacian_p(g, phi), (hu, hv, hw))


def oracle_step_rk3(g, state, f=None, re=100.0, dt=1e-3, cfl=0.0,
                    fconst=(0.0, 0.0, 0.0)):
    """One full RK3 step n -> n+1 (three sub-steps).  dt: given, or from the
    CFL rule on u^n (fixed for the three sub-steps).  The stored history
    H^{n-1} is not used (rho_1 = 0); the last sub-step's H is stored.
    Returns (new_state, stats) as oracle_step."""
    u, v, w, p = state["u"], state["v"], state["w"], state["p"]
    w = op.wall_w(g, w)
    if cfl > 0.0:
        dt = oracle_cfl_dt(g, u, v, w, cfl)
    h = (state["hu"], state["hv"], state["hw"])
    for gam, rho in zip(RK3_GAMMA, RK3_RHO):
        u, v, w, p, h = rk3_substep(g, u, v, w, p, h, dt, gam, rho, gam + rho, re, f, fconst)
    new = {"u": u, "v": v, "w": w, "p": p, "hu": h[0], "hv": h[1], "hw": h[2],
           "have_prev_h": 1}
    stats = {"dt_used": dt}
    stats.update(oracle_stats(g, u, v, w, dt))
    return new, stats
