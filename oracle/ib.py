"""Immersed-boundary forcing by moving least squares and the hydrodynamic
loads on the immersed surface (Sec. 2.1, Eq. 4 and Eqs. 5-7; Sec. 3.2).
Test infrastructure only (see package header).

The paper fixes: Lagrangian markers at the centroids of a triangulated wet
surface; a support of 3 x 3 x 3 Eulerian nodes around each marker, per
velocity component on that component's staggered points; the transfer
operators of a moving-least-squares fit with the linear basis [1, x, y, z]
and an exponential weight centred on the marker (Eq. 4); the forcing found
at the marker and spread back over the same nodes; loads from the pressure
and the viscous stress on each face (Eq. 5 two-sided, Eq. 6 one-sided), a
third of each face's load to each of its three nodes (Eq. 7).  It defers
the rest to its citations; the readings used here (and by the CUDA path):

* support: per axis the node of the component's grid nearest to the point
  and its two neighbours (periodic x, y; with walls the support must stay
  on interior nodes); a point exactly halfway between two nodes takes the
  one whose control volume, taken half-open [lower end, upper end), holds
  it (control volumes end at the faces for centre nodes and at the centres
  for face nodes);
* weight w_k = exp(-r_k^2), r_k^2 = sum_d ((x_k,d - x_d) / h_d)^2, h_d the
  extent along axis d of the nearest node's control volume (dx, dy; dz_k
  for centre points, hc_k for w faces);
* basis p(x) = [1, (x - x_b)/h_x, (y - y_b)/h_y, (z - z_b)/h_z]: the linear
  basis in coordinates centred and scaled at the evaluation point (it spans
  the same functions, so the fit is the same);
* transfer operators phi_k = w_k p(x_k)^T A^-1 p(x_b), A = sum_k w_k p(x_k)
  p(x_k)^T: the weighted least-squares linear fit evaluated at x_b;
* direct forcing: F_b = (U_b - u(x_b)) / dt per component, U_b the marker's
  prescribed velocity;
* spreading: f(x_k) += phi_k F_b dV_b / dV_k (dV_b the marker's forcing
  volume, dV_k the node's control volume dx dy dz_k for u, v and
  dx dy hc_k for w), which conserves sum(f dV) = sum(F dV_b);
* loads: pressure and velocity gradient at a probe x_f + h n_f (and
  x_f - h n_f on the other side of a two-sided face), by the same fit: the
  value is its constant coefficient, the gradient its linear coefficients
  (exact for linear fields); tau = Re^-1 (grad u + grad u^T).
"""

import numpy as np

U, V, W, P = 0, 1, 2, 3        # staggered locations: u, v, w faces, p centres


def _axis_nodes(g, loc, axis):
    """Coordinates of the component's nodes along one axis."""
    if axis == 0:
        return g.x_face() if loc == U else g.x_centre()
    if axis == 1:
        return g.y_face() if loc == V else g.y_centre()
    return g.zf[:-1] if loc == W else g.zc


def _nearest(coords, bounds, x, periodic, length):
    """Index of the node nearest to x; on a tie the node whose control
    volume [bounds[i], bounds[i+1]) holds x (periodic: x taken into the
    box first)."""
    if periodic:
        x = bounds[0] + (x - bounds[0]) % length
        d = np.abs((coords - x + 0.5 * length) % length - 0.5 * length)
    else:
        d = np.abs(coords - x)
    cand = np.flatnonzero(d == d.min())
    if len(cand) == 1:
        return int(cand[0])
    for i in cand:
        lo, hi = bounds[i], bounds[i + 1]
        if lo <= x < hi:
            return int(i)
    return int(cand[-1])


def _axis_bounds(g, loc, axis):
    """Control-volume ends of the component's nodes along one axis: faces
    for centre nodes, centres for face nodes (one more entry than nodes)."""
    if axis == 0:
        return (np.arange(g.nx + 1) - (0.5 if loc == U else 0.0)) * g.dx
    if axis == 1:
        return (np.arange(g.ny + 1) - (0.5 if loc == V else 0.0)) * g.dy
    if loc != W:
        return g.zf
    zc = g.zc
    if g.walls:
        return np.concatenate([[2 * g.zf[0] - zc[0]], zc])
    lz = g.zf[-1] - g.zf[0]
    return np.concatenate([[zc[-1] - lz], zc])


def support(g, loc, xb):
    """Indices (k, j, i) of the 27 support nodes of point xb for the
    component at staggered location loc, their coordinates relative to xb
    (periodic images taken in x, y), and the axis spacings h."""
    nodes = [_axis_nodes(g, loc, a) for a in range(3)]
    lengths = (g.lx, g.ly, g.zf[-1] - g.zf[0])
    periodic = (True, True, not g.walls)
    c = [_nearest(nodes[a], _axis_bounds(g, loc, a), xb[a], periodic[a], lengths[a])
         for a in range(3)]
    n = (g.nx, g.ny, g.nz)
    if g.walls:
        lo = 1 if loc == W else 0
        if not (lo + 1 <= c[2] <= g.nz - 2):
            raise ValueError("support of %r leaves the interior z nodes" % (xb,))
    h = [g.dx, g.dy, g.hc[c[2]] if loc == W else g.dz[c[2]]]
    idx, rel = [], []
    for dk in (-1, 0, 1):
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                ii = [c[0] + di, c[1] + dj, c[2] + dk]
                r = []
                for a in range(3):
                    m = ii[a] % n[a]
                    x = nodes[a][m]
                    d = x - xb[a]
                    if periodic[a]:
                        d = (d + 0.5 * lengths[a]) % lengths[a] - 0.5 * lengths[a]
                    ii[a] = m
                    r.append(d)
                idx.append((ii[2], ii[1], ii[0]))
                rel.append(r)
    return idx, np.array(rel), np.array(h)


def mls_fit_matrices(rel, h):
    """Weights w_k, basis rows p(x_k) (centred and scaled) and the moment
    matrix A = sum_k w_k p(x_k) p(x_k)^T of one support."""
    s = rel / h[None, :]
    w = np.exp(-(s * s).sum(axis=1))
    pk = np.hstack([np.ones((len(rel), 1)), s])
    A = (w[:, None, None] * pk[:, :, None] * pk[:, None, :]).sum(axis=0)
    return w, pk, A


def transfer(g, loc, xb):
    """Support indices and transfer operators phi_k (Eq. 4) at point xb."""
    idx, rel, h = support(g, loc, xb)
    w, pk, A = mls_fit_matrices(rel, h)
    alpha = np.linalg.solve(A, np.array([1.0, 0.0, 0.0, 0.0]))
    return idx, w * (pk @ alpha)


def fit(g, field, loc, x):
    """Value and gradient at x of the weighted least-squares linear fit of
    field (at staggered location loc) over the support of x."""
    idx, rel, h = support(g, loc, x)
    w, pk, A = mls_fit_matrices(rel, h)
    vals = np.array([field[k] for k in idx])
    a = np.linalg.solve(A, (w[:, None] * pk * vals[:, None]).sum(axis=0))
    return a[0], a[1:] / h


def node_volumes(g, loc):
    """Control volume of every node of the component: dx dy dz_k (u, v, p)
    or dx dy hc_k (w)."""
    vz = g.hc[: g.nz] if loc == W else g.dz
    return (g.dx * g.dy * vz)[:, None, None] * np.ones(g.shape)


def ib_forcing(g, u, v, w, xb, ub, dvb, dt, f=None):
    """Direct forcing of markers xb (M x 3) with prescribed velocities ub
    (M x 3) and forcing volumes dvb (M): interpolate each velocity component
    at every marker from the given fields, F_b = (U_b - u(x_b)) / dt, spread
    F_b over the same support.  Returns ((fx, fy, fz), u_interp (M x 3));
    f: fields to accumulate into (copied), else zeros."""
    fields = (u, v, w)
    out = [np.zeros(g.shape) for _ in range(3)] if f is None else [a.copy() for a in f]
    ui = np.zeros((len(xb), 3))
    vols = [node_volumes(g, c) for c in (U, V, W)]
    for c in range(3):
        for b in range(len(xb)):
            idx, phi = transfer(g, c, xb[b])
            ui[b, c] = sum(p * fields[c][k] for p, k in zip(phi, idx))
            fb = (ub[b, c] - ui[b, c]) / dt
            for p, k in zip(phi, idx):
                out[c][k] += p * fb * dvb[b] / vols[c][k]
    return tuple(out), ui


def face_loads(g, p, u, v, w, xf, nf, af, two_sided, probe, re):
    """Hydrodynamic load on each face (Eq. 6; Eq. 5 where two_sided): at the
    probe x_f + probe n_f the pressure p+ and stress tau+ = Re^-1 (grad u +
    grad u^T) from the fits; the traction -p n + tau . n times the area.
    Two-sided faces subtract the traction seen at x_f - probe n_f.  Returns
    (F (F x 3), probe pressures (F x 2), the second column 0 for one-sided
    faces)."""
    fields = (u, v, w)
    F = np.zeros((len(xf), 3))
    pp = np.zeros((len(xf), 2))
    for f in range(len(xf)):
        n = nf[f]
        trac = []
        for side, sgn in enumerate((1.0, -1.0)):
            if side == 1 and not two_sided[f]:
                break
            x = xf[f] + sgn * probe * n
            pv, _ = fit(g, p, P, x)
            grad = np.array([fit(g, fields[c], c, x)[1] for c in range(3)])  # grad[i, j] = d u_i / d x_j
            tau = (grad + grad.T) / re
            trac.append(-pv * n + tau @ n)
            pp[f, side] = pv
        t = trac[0] - trac[1] if len(trac) == 2 else trac[0]
        F[f] = t * af[f]
    return F, pp


def nodal_loads(F, tris, nnodes):
    """Eq. 7: a third of each face's load to each of its three nodes."""
    out = np.zeros((nnodes, 3))
    for f, tri in enumerate(tris):
        for n in tri:
            out[n] += F[f] / 3.0
    return out
