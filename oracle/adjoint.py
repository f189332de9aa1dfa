"""Discrete adjoint (exact transpose) of one fractional step.  Test
infrastructure only (see package header).

The step of ``step.oracle_step`` with a frozen dt (the CFL maximum is not
differentiable, so adjoint runs fix dt) maps
    (u^n, p^n, H^{n-1}, f)  ->  (u^{n+1}, p^{n+1}, H^n)
and is quadratic in u^n (through the advection term H^n = A(u^n)) and linear
in everything else.  Given cotangents of the outputs, ``oracle_adjoint_step``
returns the cotangents of the inputs, with respect to the plain Euclidean
inner product of the stored arrays (so the gradient of a functional J of the
stored values is dJ/du itself, volume weights included in J).

Every linear piece is transposed explicitly:
* G^T, D^T -- reversed difference stencils;
* the x and y sweeps and second differences are symmetric (circulant);
* the z operators are L_z = W^-1 S with S symmetric and W = diag(dz_k)
  (z centres) or diag(hc_k) (z faces), so L_z^T = W L_z W^-1 and
  (I - beta L_z)^-T = W (I - beta L_z)^-1 W^-1;
* the Poisson solve restricted to compatible right-hand sides is the
  pseudo-inverse of D G, which is self-adjoint in the V-weighted inner
  product (V = cell volumes), so its Euclidean transpose is
  V (DG)^+ V^-1 applied after removing the V-weighted mean;
* the advection Jacobian transpose is the reverse of ``operators.advection``
  term by term (products, two-point averages, differences).
"""

import numpy as np

from . import operators as op
from .poisson import oracle_poisson
from . import step as st


def _zcol(v):
    return v[:, None, None]


# ------------------------------------------------------------ transposes ----
def gradient_T(g, gu, gv, gw):
    """G^T (gu, gv, gw) at the cell centres."""
    gw = op.wall_w(g, gw)
    out = (gu - op.xp(gu)) / g.dx + (gv - op.yp(gv)) / g.dy
    c = gw / _zcol(g.hc[: g.nz])
    if g.walls:
        c[0] = 0.0
    out += c - op.zup(c, g) if g.walls else c - np.roll(c, -1, axis=0)
    return out


def divergence_T(g, s):
    """D^T s: (u-bar, v-bar, w-bar); with walls the wall face gets 0."""
    ub = (op.xm(s) - s) / g.dx
    vb = (op.ym(s) - s) / g.dy
    t = s / _zcol(g.dz)
    wb = op.zdn(t, g) - t
    if g.walls:
        wb[0] = 0.0
    return ub, vb, wb


def lapz_centre_T(g, a):
    w = _zcol(g.dz)
    return w * op.lapz_centre(g, a / w)


def lapz_face_T(g, a):
    w = _zcol(g.hc[: g.nz])
    a = op.wall_w(g, a)
    out = w * op.lapz_face(g, a / w)
    if g.walls:
        out[0] = 0.0
    return out


def viscous_T(g, au, av, aw):
    return (op.lap_xy(g, au) + lapz_centre_T(g, au),
            op.lap_xy(g, av) + lapz_centre_T(g, av),
            op.wall_w(g, op.lap_xy(g, op.wall_w(g, aw))) + lapz_face_T(g, aw))


def laplacian_p_T(g, a):
    w = _zcol(g.dz)
    return op.lap_xy(g, a) + w * op.lapz_poisson(g, a / w)


def sweeps_T(g, beta, bu, bv, bw):
    """(S_z S_y S_x)^T = S_x^T S_y^T S_z^T, S_d = (I - beta L_d)^-1."""
    wc = _zcol(g.dz)
    wf = _zcol(g.hc[: g.nz])
    ru = wc * st.sweep_z_centre(g, beta, bu / wc)
    rv = wc * st.sweep_z_centre(g, beta, bv / wc)
    bw = op.wall_w(g, bw)
    rw = wf * st.sweep_z_face(g, beta, bw / wf)
    if g.walls:
        rw[0] = 0.0
    out = []
    for r in (ru, rv, rw):
        out.append(st.sweep_x(g, beta, st.sweep_y(g, beta, r)))
    if g.walls:
        out[2][0] = 0.0
    return tuple(out)


def poisson_T(g, phib):
    """Transpose of s -> phi restricted to compatible s: V P(compat(phib / V))."""
    vol = np.broadcast_to(g.cell_volume_uvp(), g.shape)
    x = phib / vol
    x = x - phib.sum() / vol.sum()
    return vol * oracle_poisson(g, x)


def advection_T(g, u, v, w, bu, bv, bw):
    """J_A(u)^T applied to (bu, bv, bw): the reverse of operators.advection."""
    w = op.wall_w(g, w)
    nz = g.nz
    dz = _zcol(g.dz)
    hc = _zcol(g.hc[:nz])
    a, b, c = -bu, -bv, -bw.copy()
    if g.walls:
        c[0] = 0.0
    # forward intermediates
    uc = 0.5 * (u + op.xp(u))
    vc = 0.5 * (v + op.yp(v))
    wc = 0.5 * (w + op.zup(w, g))
    vx = 0.5 * (v + op.xm(v))
    uy = 0.5 * (u + op.ym(u))
    wx = 0.5 * (w + op.xm(w))
    uz = 0.5 * (u + op.zdn(u, g))
    wy = 0.5 * (w + op.ym(w))
    vz = 0.5 * (v + op.zdn(v, g))
    # cotangents of the fluxes
    qb = (a - op.xp(a)) / g.dx                       # of uc^2
    rb = (b - op.yp(b)) / g.dy                       # of vc^2
    sb = c / hc - np.roll(c / hc, -1, axis=0)        # of wc^2
    euv = (op.ym(a) - a) / g.dy + (op.xm(b) - b) / g.dx
    euw = np.zeros((nz + 1,) + u.shape[1:])
    evw = np.zeros((nz + 1,) + u.shape[1:])
    euw[1:] += a / dz
    euw[:-1] -= a / dz
    evw[1:] += b / dz
    evw[:-1] -= b / dz
    euw[:nz] += (op.xm(c) - c) / g.dx
    evw[:nz] += (op.ym(c) - c) / g.dy
    if g.walls:
        euw[0] = 0.0
        evw[0] = 0.0
    else:
        euw[0] += euw[nz]
        evw[0] += evw[nz]
    euw = euw[:nz]
    evw = evw[:nz]
    # back to the velocities
    ucb = 2.0 * uc * qb
    vcb = 2.0 * vc * rb
    wcb = 2.0 * wc * sb
    ub = 0.5 * (ucb + op.xm(ucb))
    vb = 0.5 * (vcb + op.ym(vcb))
    wb = 0.5 * (wcb + op.zdn(wcb, g))
    vxb, uyb = euv * uy, euv * vx
    vb += 0.5 * (vxb + op.xp(vxb))
    ub += 0.5 * (uyb + op.yp(uyb))
    wxb, uzb = euw * uz, euw * wx
    wb += 0.5 * (wxb + op.xp(wxb))
    ub += 0.5 * (uzb + op.zup(uzb, g))
    wyb, vzb = evw * vz, evw * wy
    wb += 0.5 * (wyb + op.yp(wyb))
    vb += 0.5 * (vzb + op.zup(vzb, g))
    if g.walls:
        wb[0] = 0.0
    return ub, vb, wb


# ------------------------------------------------------------ step adjoint --
def oracle_adjoint_step(g, state, cot, f=None, re=100.0, dt=1e-3, gamma=1.5,
                        rho=-0.5):
    """Cotangents of the step inputs.  `state` holds the forward inputs u, v,
    w (of step n) and have_prev_h; `cot` holds the cotangents of the outputs:
    u, v, w, p (of step n+1) and hu, hv, hw (of the stored history H^n).
    Returns a dict with u, v, w, p (of step n), hu, hv, hw (of H^{n-1}) and
    fx, fy, fz (of the body force)."""
    if not state.get("have_prev_h", 0):
        gamma, rho = 1.0, 0.0
    beta = dt / (2.0 * re)
    u, v, w = state["u"], state["v"], op.wall_w(g, state["w"])
    ubar, vbar, wbar = cot["u"], cot["v"], op.wall_w(g, cot["w"])
    pbar = cot["p"]
    # u^{n+1} = u* - dt G phi ; p^{n+1} = p^n + phi - beta DG phi
    phib = -dt * gradient_T(g, ubar, vbar, wbar) + pbar - beta * laplacian_p_T(g, pbar)
    sb = poisson_T(g, phib)
    du, dv, dw = divergence_T(g, sb)
    us_b = ubar + du / dt
    vs_b = vbar + dv / dt
    ws_b = wbar + dw / dt
    # u* = u^n + S RHS
    ru, rv, rw = sweeps_T(g, beta, us_b, vs_b, ws_b)
    # RHS = dt[gamma H^n + rho H^{n-1} + Re^-1 L u^n - G p^n + f]
    hbu = dt * gamma * ru + cot["hu"]
    hbv = dt * gamma * rv + cot["hv"]
    hbw = op.wall_w(g, dt * gamma * rw + cot["hw"])
    lu, lv, lw = viscous_T(g, ru, rv, rw)
    au, av, aw = advection_T(g, u, v, w, hbu, hbv, hbw)
    out = {
        "u": us_b + dt / re * lu + au,
        "v": vs_b + dt / re * lv + av,
        "w": op.wall_w(g, ws_b + dt / re * lw + aw),
        "p": pbar - dt * gradient_T(g, ru, rv, rw),
        "hu": dt * rho * ru, "hv": dt * rho * rv, "hw": op.wall_w(g, dt * rho * rw),
        "fx": dt * ru, "fy": dt * rv, "fz": op.wall_w(g, dt * rw),
    }
    return out
