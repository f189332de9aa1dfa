"""Shear-thinning (Carreau-Yasuda) blood rheology (Sec. 2.1: the viscous
stress depends on the strain rate E = (grad u + grad u^T) / 2 through the
Carreau-Yasuda law; the Newtonian tau = 2 Re^-1 E is the special case the
code selects by a flag).  Test infrastructure only (see package header).

The paper names the law and defers its form, parameters and time treatment
to its citations.  The readings used here (and by the CUDA path):

* tau = 2 Re^-1 eta(gdot) E, Re built on the zero-shear viscosity, with
  eta(gdot) = eta_inf + (1 - eta_inf) (1 + (lam gdot)^a)^((n - 1) / a),
  gdot = sqrt(2 E:E); lam, n, a, eta_inf are given by the caller;
* time treatment: the Newtonian part Re^-1 L u stays in the implicit
  Crank-Nicolson sweeps; the remainder div(2 Re^-1 (eta - 1) E) is explicit
  and joins the advection term H (so it takes the same Adams-Bashforth
  weights and is stored in the history); eta <= 1, so the implicit part
  carries the largest viscosity;
* discrete strain rate on the staggered mesh: normal components at the cell
  centres (E_xx = (u_{i+1} - u_i) / dx, ...), shear components at the cell
  edges where the advection's cross fluxes live (E_xy at (x_i, y_j, zc_k),
  E_xz at (x_i, y_{j+1/2}, z_k), E_yz at (x_{i+1/2}, y_j, z_k)), each the
  half sum of the two cross differences (z differences over hc_k, the wall
  value of a tangential velocity 0 and w = 0 on the walls);
* gdot at each cell centre from its normal components and the averages of
  its four surrounding edges of each shear kind; eta at the centres; the
  excess viscosity (eta - 1) / Re at an edge is the average over the cells
  around it (four, or the two on the fluid side of a wall edge);
* the explicit term at each component's points is the divergence of
  tau' = 2 nu' E, nu' = (eta - 1) / Re, with the differences of the
  Newtonian operators (dx, dy; dz_k at centres, hc_k at w faces).
"""

import numpy as np

from . import operators as op


def carreau_yasuda(gdot, lam, n, a, eta_inf):
    """Viscosity relative to the zero-shear one."""
    return eta_inf + (1.0 - eta_inf) * (1.0 + (lam * gdot) ** a) ** ((n - 1.0) / a)


def strain_rates(g, u, v, w):
    """(Exx, Eyy, Ezz) at the centres [nz, ny, nx]; Exy at the xy edges
    [nz, ny, nx]; Exz, Eyz at the xz, yz edges [nz + 1, ny, nx] (edge k at
    the face z_k; with periodic z row nz repeats row 0)."""
    w = op.wall_w(g, w)
    nz = g.nz
    exx = (op.xp(u) - u) / g.dx
    eyy = (op.yp(v) - v) / g.dy
    ezz = (op.zup(w, g) - w) / g.dz[:, None, None]
    exy = 0.5 * ((u - op.ym(u)) / g.dy + (v - op.xm(v)) / g.dx)
    hc = g.hc[:, None, None]
    exz = np.empty((nz + 1,) + u.shape[1:])
    eyz = np.empty((nz + 1,) + u.shape[1:])
    wx = (w - op.xm(w)) / g.dx          # at face k (xz edge)
    wy = (w - op.ym(w)) / g.dy          # at face k (yz edge)
    exz[:nz] = 0.5 * ((u - op.zdn(u, g)) / hc[:nz] + wx)
    eyz[:nz] = 0.5 * ((v - op.zdn(v, g)) / hc[:nz] + wy)
    if g.walls:
        # the top wall edge: the tangential velocity above is 0 and w = 0
        exz[nz] = 0.5 * (0.0 - u[nz - 1]) / hc[nz]
        eyz[nz] = 0.5 * (0.0 - v[nz - 1]) / hc[nz]
    else:
        exz[nz] = exz[0]
        eyz[nz] = eyz[0]
    return (exx, eyy, ezz), exy, exz, eyz


def shear_rate(g, normal, exy, exz, eyz):
    """gdot = sqrt(2 E:E) at the cell centres, the shear components averaged
    from the four edges around each centre."""
    exx, eyy, ezz = normal
    exy_c = 0.25 * (exy + op.xp(exy) + op.yp(exy) + op.xp(op.yp(exy)))
    exz_c = 0.25 * (exz[:-1] + exz[1:] + op.xp(exz[:-1]) + op.xp(exz[1:]))
    eyz_c = 0.25 * (eyz[:-1] + eyz[1:] + op.yp(eyz[:-1]) + op.yp(eyz[1:]))
    ee = exx ** 2 + eyy ** 2 + ezz ** 2 + 2.0 * (exy_c ** 2 + exz_c ** 2 + eyz_c ** 2)
    return np.sqrt(2.0 * ee)


def excess_viscosity_edges(g, nu):
    """nu' at the xy, xz, yz edges from the centre values: the average of
    the cells around each edge (two at a wall edge)."""
    nz = g.nz
    nu_xy = 0.25 * (nu + op.xm(nu) + op.ym(nu) + op.xm(op.ym(nu)))
    nx_avg = 0.5 * (nu + op.xm(nu))      # x average at (x_i, y_{j+1/2}, zc_k)
    ny_avg = 0.5 * (nu + op.ym(nu))      # y average at (x_{i+1/2}, y_j, zc_k)
    nu_xz = np.empty((nz + 1,) + nu.shape[1:])
    nu_yz = np.empty((nz + 1,) + nu.shape[1:])
    if g.walls:
        nu_xz[1:nz] = 0.5 * (nx_avg[1:] + nx_avg[:-1])
        nu_yz[1:nz] = 0.5 * (ny_avg[1:] + ny_avg[:-1])
        nu_xz[0], nu_xz[nz] = nx_avg[0], nx_avg[nz - 1]
        nu_yz[0], nu_yz[nz] = ny_avg[0], ny_avg[nz - 1]
    else:
        nu_xz[:nz] = 0.5 * (nx_avg + np.roll(nx_avg, 1, axis=0))
        nu_yz[:nz] = 0.5 * (ny_avg + np.roll(ny_avg, 1, axis=0))
        nu_xz[nz], nu_yz[nz] = nu_xz[0], nu_yz[0]
    return nu_xy, nu_xz, nu_yz


def stress_divergence(g, u, v, w, nu_c, nu_xy, nu_xz, nu_yz):
    """div(2 nu E) at the u, v, w points for given viscosities at the
    centres and edges (Hw[0] = 0 with walls)."""
    (exx, eyy, ezz), exy, exz, eyz = strain_rates(g, u, v, w)
    txx, tyy, tzz = 2 * nu_c * exx, 2 * nu_c * eyy, 2 * nu_c * ezz
    txy, txz, tyz = 2 * nu_xy * exy, 2 * nu_xz * exz, 2 * nu_yz * eyz
    dz = g.dz[:, None, None]
    hx = ((txx - op.xm(txx)) / g.dx + (op.yp(txy) - txy) / g.dy
          + (txz[1:] - txz[:-1]) / dz)
    hy = ((op.xp(txy) - txy) / g.dx + (tyy - op.ym(tyy)) / g.dy
          + (tyz[1:] - tyz[:-1]) / dz)
    hc = g.hc[: g.nz, None, None]
    hz = ((op.xp(txz[:-1]) - txz[:-1]) / g.dx + (op.yp(tyz[:-1]) - tyz[:-1]) / g.dy
          + (tzz - np.roll(tzz, 1, axis=0)) / hc)
    if g.walls:
        hz[0] = 0.0
    return hx, hy, hz


def non_newtonian_term(g, u, v, w, re, lam, n, a, eta_inf):
    """The explicit remainder div(2 Re^-1 (eta(gdot) - 1) E) at the u, v, w
    points."""
    normal, exy, exz, eyz = strain_rates(g, u, v, w)
    gdot = shear_rate(g, normal, exy, exz, eyz)
    nu = (carreau_yasuda(gdot, lam, n, a, eta_inf) - 1.0) / re
    return stress_divergence(g, u, v, w, nu, *excess_viscosity_edges(g, nu))
