"""Discrete operators of the staggered second-order scheme (Sec. 2.1: central
second-order finite differences on a staggered mesh, Eq. 2 with the Newtonian
stress tau = 2 Re^-1 E, whose divergence for a solenoidal field is
Re^-1 lap(u)).  Test infrastructure only (see package header).

Arrays are ``a[k, j, i]``; x and y are periodic (np.roll), z is either
periodic or bounded by no-slip walls (explicit boundary handling below).
With walls the stored w[0] is the bottom wall value and must be 0.

Readings of points the paper leaves to its citations:
* advection is written in divergence form, -div(uu), with arithmetic two-point
  averages to the flux points (cell centres for the normal fluxes, cell edges
  for the cross fluxes); on a stretched z the cross-flux average of two
  z-centre values is the plain arithmetic mean;
* tangential velocities see a Dirichlet zero at the wall, half a cell
  (dz_0/2) below the first centre;
* the Poisson operator is the compound D G, whose wall rows lose the wall flux
  (the wall-normal velocity at the walls is fixed, so the pressure gradient
  there never acts).
"""

import numpy as np


# ----------------------------------------------------------------- shifts ---
def xp(a):
    """a[..., i+1] (periodic)."""
    return np.roll(a, -1, axis=2)


def xm(a):
    """a[..., i-1] (periodic)."""
    return np.roll(a, 1, axis=2)


def yp(a):
    return np.roll(a, -1, axis=1)


def ym(a):
    return np.roll(a, 1, axis=1)


def zdn(a, g):
    """a[k-1]; with walls the value below k = 0 is 0."""
    if g.walls:
        out = np.empty_like(a)
        out[1:] = a[:-1]
        out[0] = 0.0
        return out
    return np.roll(a, 1, axis=0)


def zup(a, g):
    """a[k+1]; with walls the value above k = nz-1 is 0."""
    if g.walls:
        out = np.empty_like(a)
        out[:-1] = a[1:]
        out[-1] = 0.0
        return out
    return np.roll(a, -1, axis=0)


def _zcol(v):
    return v[:, None, None]


def wall_w(g, w):
    """w with the bottom-wall face forced to its boundary value 0."""
    if g.walls:
        w = w.copy()
        w[0] = 0.0
    return w


# -------------------------------------------------------------- advection ---
def advection(g, u, v, w):
    """H = -div(u u) at each component's own staggered points (the convective
    term of Eq. 2/Eq. 3, moved to the right-hand side).

    H_u = -[ d_x(U U) + d_y(V^x U^y) + d_z(W^x U^z) ]
    H_v = -[ d_x(U^y V^x) + d_y(V V) + d_z(W^y V^z) ]
    H_w = -[ d_x(U^z W^x) + d_y(V^z W^y) + d_z(W W) ]

    where a^x is the two-point average in x to the flux point.  Returns
    (Hu, Hv, Hw); with walls Hw[0] = 0 (the wall face carries no unknown).
    """
    w = wall_w(g, w)
    dx, dy = g.dx, g.dy
    dz = _zcol(g.dz)
    nz = g.nz

    # normal fluxes at cell centres
    uc = 0.5 * (u + xp(u))             # u at (x_{i+1/2}, y_{j+1/2}, zc_k)
    vc = 0.5 * (v + yp(v))
    wc = 0.5 * (w + zup(w, g))         # w at cell centre k (w[nz] = 0 / wraps)

    # xy edges at (x_i, y_j, zc_k): v averaged in x times u averaged in y
    e_uv = (0.5 * (v + xm(v))) * (0.5 * (u + ym(u)))

    # xz edges at (x_i, y_{j+1/2}, z_k), k = 0..nz (one extra top edge)
    # yz edges at (x_{i+1/2}, y_j, z_k)
    e_uw = np.empty((nz + 1,) + u.shape[1:])
    e_vw = np.empty((nz + 1,) + u.shape[1:])
    e_uw[:nz] = (0.5 * (w + xm(w))) * (0.5 * (u + zdn(u, g)))
    e_vw[:nz] = (0.5 * (w + ym(w))) * (0.5 * (v + zdn(v, g)))
    if g.walls:
        e_uw[0] = 0.0
        e_uw[nz] = 0.0
        e_vw[0] = 0.0
        e_vw[nz] = 0.0
    else:
        e_uw[nz] = e_uw[0]
        e_vw[nz] = e_vw[0]

    hu = -((uc * uc - xm(uc * uc)) / dx
           + (yp(e_uv) - e_uv) / dy
           + (e_uw[1:] - e_uw[:-1]) / dz)
    hv = -((xp(e_uv) - e_uv) / dx
           + (vc * vc - ym(vc * vc)) / dy
           + (e_vw[1:] - e_vw[:-1]) / dz)
    # w faces: the outer z difference spans two centres, distance hc_k
    hc = _zcol(g.hc[:nz])
    wc2 = wc * wc
    hw = -((xp(e_uw[:nz]) - e_uw[:nz]) / dx
           + (yp(e_vw[:nz]) - e_vw[:nz]) / dy
           + (wc2 - np.roll(wc2, 1, axis=0)) / hc)
    if g.walls:
        hw[0] = 0.0
    return hu, hv, hw


# --------------------------------------------------------------- Laplacians -
def lap_xy(g, a):
    """Periodic second differences in x and y (any staggered location)."""
    return ((xp(a) - 2.0 * a + xm(a)) / g.dx ** 2
            + (yp(a) - 2.0 * a + ym(a)) / g.dy ** 2)


def lapz_centre(g, a):
    """d2/dz2 at z-centre points (u, v): fluxes at faces over hc, difference
    over dz.  Walls: Dirichlet 0 at the wall, hc_0 = dz_0/2 away."""
    nz = g.nz
    flux = np.empty((nz + 1,) + a.shape[1:])
    hc = _zcol(g.hc)
    flux[1:nz] = (a[1:] - a[:-1]) / hc[1:nz]
    if g.walls:
        flux[0] = a[0] / hc[0]
        flux[nz] = -a[nz - 1] / hc[nz]
    else:
        flux[0] = (a[0] - a[nz - 1]) / hc[0]
        flux[nz] = flux[0]
    return (flux[1:] - flux[:-1]) / _zcol(g.dz)


def lapz_face(g, w):
    """d2/dz2 at w faces: fluxes at centres over dz, difference over hc.
    Walls: w = 0 on both wall faces; the result at the wall face is 0."""
    w = wall_w(g, w)
    flux = (zup(w, g) - w) / _zcol(g.dz)          # at centre k
    out = (flux - np.roll(flux, 1, axis=0)) / _zcol(g.hc[: g.nz])
    if g.walls:
        out[0] = 0.0
    return out


def lapz_poisson(g, phi):
    """z part of the compound operator D G at centres.  Walls: Neumann (the
    gradient at the wall faces is not used, the flux there is dropped)."""
    nz = g.nz
    flux = np.empty((nz + 1,) + phi.shape[1:])
    hc = _zcol(g.hc)
    flux[1:nz] = (phi[1:] - phi[:-1]) / hc[1:nz]
    if g.walls:
        flux[0] = 0.0
        flux[nz] = 0.0
    else:
        flux[0] = (phi[0] - phi[nz - 1]) / hc[0]
        flux[nz] = flux[0]
    return (flux[1:] - flux[:-1]) / _zcol(g.dz)


def viscous(g, u, v, w):
    """L applied to each velocity component (the Newtonian viscous term of
    Eq. 2 is Re^-1 times this)."""
    return (lap_xy(g, u) + lapz_centre(g, u),
            lap_xy(g, v) + lapz_centre(g, v),
            lap_xy(g, wall_w(g, w)) + lapz_face(g, w))


def laplacian_p(g, phi):
    """Compound Laplacian D G at cell centres."""
    return lap_xy(g, phi) + lapz_poisson(g, phi)


# ------------------------------------------------------ gradient / divergence
def gradient(g, p):
    """G p at the u, v, w points; with walls the wall face gets 0."""
    gx = (p - xm(p)) / g.dx
    gy = (p - ym(p)) / g.dy
    gz = (p - np.roll(p, 1, axis=0)) / _zcol(g.hc[: g.nz])
    if g.walls:
        gz[0] = 0.0
    return gx, gy, gz


def divergence(g, u, v, w):
    """D u at cell centres; with walls w = 0 on both wall faces."""
    w = wall_w(g, w)
    return ((xp(u) - u) / g.dx + (yp(v) - v) / g.dy
            + (zup(w, g) - w) / _zcol(g.dz))
