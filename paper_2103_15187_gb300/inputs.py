"""Seeded synthetic inputs for the fractional-step solver.

This module builds initial velocity fields and body forces shaped like the
workloads of the FSEI paper (arXiv 2103.15187): a Taylor-Green vortex on a
triply periodic box, a wall-bounded channel (periodic x, y; no-slip walls at
z = +-1 with a tanh-stretched z mesh) with a laminar Poiseuille profile plus a
divergence-free random perturbation, and a field of Gaussian force blobs that
stands in for the immersed-boundary forcing.  It holds none of the solver's
arithmetic: it only samples analytic functions at the staggered points and
takes a discrete curl of a random vector potential so that the perturbation is
exactly (to round-off) divergence-free on the staggered mesh.

Everything is float64 numpy, drawn from numpy's PCG64 with an explicit seed.
Arrays are ``a[k, j, i]`` (x fastest).  Staggering: u at (x_i, y_{j+1/2},
zc_k), v at (x_{i+1/2}, y_j, zc_k), w at (x_{i+1/2}, y_{j+1/2}, z_k),
p at the centres; with walls w[0] is the (zero) bottom wall face.
"""

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

Z_PERIODIC = 0
Z_WALLS = 1


@dataclass
class Case:
    """One synthetic workload: grid description, initial state, force and
    step parameters (plain data, consumed by both the library binding and the
    tests)."""
    name: str
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    zbc: int
    lz: float
    stretch: float
    re: float
    dt: float
    cfl: float
    nsteps: int
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    p: np.ndarray
    f: Optional[tuple] = None
    fconst: tuple = (0.0, 0.0, 0.0)
    extra: dict = field(default_factory=dict)

    @property
    def cells(self):
        return self.nx * self.ny * self.nz


def z_faces(nz, zbc, lz=2.0, stretch=0.0):
    """z faces z_0..z_nz.  Walls: z in [-1, 1], tanh clustering
    z_k = tanh(s(2k/nz - 1))/tanh(s) (uniform when s = 0).  Periodic: uniform
    on [0, lz)."""
    k = np.arange(nz + 1, dtype=np.float64)
    if zbc == Z_PERIODIC:
        return k * (lz / nz)
    if stretch > 0.0:
        return np.tanh(stretch * (2.0 * k / nz - 1.0)) / np.tanh(stretch)
    return -1.0 + 2.0 * k / nz


def _zc(zf):
    return 0.5 * (zf[1:] + zf[:-1])


# ------------------------------------------------------------ Taylor-Green --
def taylor_green(n=32, length=2.0 * np.pi, amp=1.0):
    """u = A sin x cos y cos z, v = -A cos x sin y cos z, w = 0 sampled at the
    staggered points of an n^3 periodic box of side `length`."""
    h = length / n
    xf = np.arange(n) * h
    xc = xf + 0.5 * h
    zc = xc
    u = amp * (np.cos(zc)[:, None, None] * np.cos(xc)[None, :, None]
               * np.sin(xf)[None, None, :])
    v = -amp * (np.cos(zc)[:, None, None] * np.sin(xf)[None, :, None]
                * np.cos(xc)[None, None, :])
    w = np.zeros((n, n, n))
    return u, v, w


# ----------------------------------------------- random solenoidal field ----
def _random_plane_fields(rng, nx, ny, lx, ly, kmin, kmax, slope, count):
    """`count` random real 2-D Fourier sums over integer (kx, ky) with
    kmin <= |k| <= kmax (|k| in units of 2 pi / L of each direction), mode
    amplitude |k_phys|^slope, uniform random phase.  Returned as complex
    spectra on the (ny, nx) FFT grid so callers can shift them to any
    staggered location."""
    ky = np.fft.fftfreq(ny, 1.0 / ny)[:, None]
    kx = np.fft.fftfreq(nx, 1.0 / nx)[None, :]
    kmag = np.sqrt(kx ** 2 + ky ** 2)
    sel = (kmag >= kmin) & (kmag <= kmax)
    kphys = np.sqrt((2 * np.pi * kx / lx) ** 2 + (2 * np.pi * ky / ly) ** 2)
    amp = np.where(sel, np.maximum(kphys, 1e-30) ** slope, 0.0)
    spectra = []
    for _ in range(count):
        z = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
        spectra.append(z * amp)
    return spectra


def _eval_plane(spec, nx, ny, sx, sy):
    """Real part of sum_k spec_k exp(i 2 pi (kx (i+sx)/nx + ky (j+sy)/ny))."""
    ky = np.fft.fftfreq(ny, 1.0 / ny)[:, None]
    kx = np.fft.fftfreq(nx, 1.0 / nx)[None, :]
    shift = np.exp(2j * np.pi * (kx * sx / nx + ky * sy / ny))
    return np.real(np.fft.ifft2(spec * shift)) * (nx * ny)


def solenoidal_field(rng, nx, ny, nz, lx, ly, zf, zbc, kmin, kmax, slope,
                     mmax=8, rms=1.0):
    """Divergence-free velocity u = curl_h A on the staggered mesh, A an
    edge-located vector potential
        A_x at (x_{i+1/2}, y_j, z_k), A_y at (x_i, y_{j+1/2}, z_k),
        A_z at (x_i, y_j, zc_k),
    A_c = sum_m P_m(z) F_{c,m}(x, y), F random horizontal Fourier sums with
    amplitude |k|^slope, P_m z profiles: with walls (1-z^2)^2 cos/sin(m pi
    (z+1)/2), m = 0..mmax (vanishing at the walls, so w = 0 there); periodic
    z: cos/sin(2 pi m z / lz).  The discrete curl uses the mesh's own
    differences, so D u vanishes to round-off.  Rescaled to the given RMS of
    all three components."""
    dx, dy = lx / nx, ly / ny
    dz = zf[1:] - zf[:-1]
    zc = _zc(zf)
    lz = zf[-1] - zf[0]

    def profiles(z):
        out = []
        for m in range(mmax + 1):
            if zbc == Z_WALLS:
                env = (1.0 - z ** 2) ** 2
                out.append(env * np.cos(m * np.pi * (z + 1.0) / 2.0))
                if m > 0:
                    out.append(env * np.sin(m * np.pi * (z + 1.0) / 2.0))
            else:
                out.append(np.cos(2 * np.pi * m * (z - zf[0]) / lz))
                if m > 0:
                    out.append(np.sin(2 * np.pi * m * (z - zf[0]) / lz))
        return out

    pf = profiles(zf)            # at faces, nz+1
    pc = profiles(zc)            # at centres, nz
    nprof = len(pf)
    # A amplitude = velocity amplitude / |k|
    spx = _random_plane_fields(rng, nx, ny, lx, ly, kmin, kmax, slope - 1.0,
                               nprof)
    spy = _random_plane_fields(rng, nx, ny, lx, ly, kmin, kmax, slope - 1.0,
                               nprof)
    spz = _random_plane_fields(rng, nx, ny, lx, ly, kmin, kmax, slope - 1.0,
                               nprof)
    # A(z, x, y) = sum_m P_m(z) F_m(x, y): one matrix product per component
    pfm = np.stack(pf, axis=1)                      # [nz+1, nprof]
    pcm = np.stack(pc, axis=1)                      # [nz, nprof]
    fx_ = np.stack([_eval_plane(spx[m], nx, ny, 0.5, 0.0).ravel() for m in range(nprof)])
    fy_ = np.stack([_eval_plane(spy[m], nx, ny, 0.0, 0.5).ravel() for m in range(nprof)])
    fz_ = np.stack([_eval_plane(spz[m], nx, ny, 0.0, 0.0).ravel() for m in range(nprof)])
    ax = (pfm @ fx_).reshape(nz + 1, ny, nx)
    ay = (pfm @ fy_).reshape(nz + 1, ny, nx)
    az = (pcm @ fz_).reshape(nz, ny, nx)
    if zbc == Z_WALLS:
        ax[0] = ax[nz] = 0.0
        ay[0] = ay[nz] = 0.0
    dzc = dz[:, None, None]
    u = (np.roll(az, -1, axis=1) - az) / dy - (ay[1:] - ay[:-1]) / dzc
    v = (ax[1:] - ax[:-1]) / dzc - (np.roll(az, -1, axis=2) - az) / dx
    w = ((np.roll(ay[:nz], -1, axis=2) - ay[:nz]) / dx
         - (np.roll(ax[:nz], -1, axis=1) - ax[:nz]) / dy)
    if zbc == Z_WALLS:
        w[0] = 0.0
    cur = np.sqrt((np.mean(u * u) + np.mean(v * v) + np.mean(w * w)) / 3.0)
    s = rms / cur
    return u * s, v * s, w * s


def gaussian_blobs(rng, nx, ny, nz, nblobs=20, sigma=8.0, amp=10.0,
                   zbc=Z_WALLS, cut=5.0):
    """Body force made of `nblobs` Gaussian blobs in index space (width sigma
    cells, periodic minimum image in x and y), each pointing in a random unit
    direction with the given amplitude; centres at least 3 sigma from the
    walls.  Each blob is truncated to the box |d| <= cut*sigma per axis
    (exp(-12.5) ~ 4e-6 of its peak at the edge).  Sampled at the u, v, w
    points; returns (fx, fy, fz)."""
    fx = np.zeros((nz, ny, nx))
    fy = np.zeros((nz, ny, nx))
    fz = np.zeros((nz, ny, nx))
    lo = 3.0 * sigma if zbc == Z_WALLS else 0.0
    hi = nz - 3.0 * sigma if zbc == Z_WALLS else float(nz)
    if hi < lo:                      # box thinner than 6 sigma: centre plane
        lo = hi = 0.5 * nz
    r = int(np.ceil(cut * sigma))
    for _ in range(nblobs):
        c = np.array([rng.uniform(0, nx), rng.uniform(0, ny),
                      rng.uniform(lo, hi)])
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        for comp, (arr, (sx, sy, sz)) in enumerate(
                ((fx, (0.0, 0.5, 0.5)), (fy, (0.5, 0.0, 0.5)),
                 (fz, (0.5, 0.5, 0.0)))):
            ii = np.arange(int(np.floor(c[0])) - r, int(np.floor(c[0])) + r + 1)
            jj = np.arange(int(np.floor(c[1])) - r, int(np.floor(c[1])) + r + 1)
            kk = np.arange(max(int(np.floor(c[2])) - r, 0),
                           min(int(np.floor(c[2])) + r + 1, nz))
            ex = np.exp(-((ii + sx - c[0]) ** 2) / (2 * sigma ** 2))
            ey = np.exp(-((jj + sy - c[1]) ** 2) / (2 * sigma ** 2))
            ez = np.exp(-((kk + sz - c[2]) ** 2) / (2 * sigma ** 2))
            blob = amp * d[comp] * (ez[:, None, None] * ey[None, :, None]
                                    * ex[None, None, :])
            if zbc == Z_WALLS and comp == 2:
                blob[kk == 0] = 0.0
            np.add.at(arr, (kk[:, None, None], (jj % ny)[None, :, None],
                            (ii % nx)[None, None, :]), blob)
    return fx, fy, fz


# ---------------------------------------------------------------- cases -----
def case_taylor_green(n=32, steps=10, re=100.0, dt=1e-3, amp=1.0):
    """Triply periodic Taylor-Green box of side 2 pi, zero body force."""
    u, v, w = taylor_green(n, 2 * np.pi, amp)
    return Case("taylor_green_%d" % n, n, n, n, 2 * np.pi, 2 * np.pi,
                Z_PERIODIC, 2 * np.pi, 0.0, re, dt, 0.0, steps, u, v, w,
                np.zeros_like(u))


def case_channel(nx=256, ny=256, nz=256, lx=2 * np.pi, ly=np.pi,
                 stretch=2.0, re=2000.0, cfl=0.5, steps=100, kmin=1.0,
                 kmax=8.0, slope=0.0, rms=0.1, seed=2, blobs=None,
                 name=None):
    """Wall-bounded channel: Poiseuille u = 1 - z^2 plus a solenoidal random
    perturbation (horizontal |k| in [kmin, kmax], velocity amplitude
    |k|^slope, RMS `rms`), uniform drive f_x = 2/Re; optional Gaussian-blob
    body force (dict of gaussian_blobs arguments)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    zf = z_faces(nz, Z_WALLS, 2.0, stretch)
    zc = _zc(zf)
    up, vp, wp = solenoidal_field(rng, nx, ny, nz, lx, ly, zf, Z_WALLS, kmin,
                                  kmax, slope, rms=rms)
    u = (1.0 - zc ** 2)[:, None, None] + up
    f = None
    if blobs is not None:
        f = gaussian_blobs(rng, nx, ny, nz, zbc=Z_WALLS, **blobs)
    return Case(name or "channel_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, lx, ly,
                Z_WALLS, 2.0, stretch, re, 0.0, cfl, steps, u, vp, wp,
                np.zeros_like(u), f, (2.0 / re, 0.0, 0.0))


def case_heart_scale(nx=512, ny=512, nz=768, steps=50, seed=3):
    """Heart-scale box: periodic x, y of length 2*96/156, stretched walls in z,
    Re = 3000, CFL 0.5, solenoidal field with |k| <= 32 and a k^-5/3 energy
    spectrum (velocity-mode amplitude k^-11/6), unit RMS, plus 20 Gaussian
    force blobs (sigma 8 cells, amplitude 10)."""
    lxy = 2.0 * 96.0 / 156.0
    rng = np.random.Generator(np.random.PCG64(seed))
    zf = z_faces(nz, Z_WALLS, 2.0, 2.0)
    u, v, w = solenoidal_field(rng, nx, ny, nz, lxy, lxy, zf, Z_WALLS, 1.0,
                               32.0, -11.0 / 6.0, rms=1.0)
    f = gaussian_blobs(rng, nx, ny, nz, zbc=Z_WALLS)
    return Case("heart_scale_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, lxy, lxy,
                Z_WALLS, 2.0, 2.0, 3000.0, 0.0, 0.5, steps, u, v, w,
                np.zeros_like(u), f)


def case_periodic_random(n=32, seed=0, re=1000.0, cfl=0.5, steps=100,
                         ke_target=0.25, ny=None, nz=None):
    """Triply periodic 2 pi box with a solenoidal random field (|k| in [1, 8])
    scaled to the Taylor-Green kinetic energy (mean |u|^2 = ke_target).  With
    ny or nz given the box is n x ny x nz cells of the same spacing 2 pi / n
    (lengths 2 pi ny / n, 2 pi nz / n)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    ly, lz = 2 * np.pi * ny / n, 2 * np.pi * nz / n
    zf = z_faces(nz, Z_PERIODIC, lz)
    u, v, w = solenoidal_field(rng, n, ny, nz, 2 * np.pi, ly, zf,
                               Z_PERIODIC, 1.0, 8.0, 0.0, rms=1.0)
    s = np.sqrt(ke_target / np.mean(u * u + v * v + w * w))
    name = ("periodic_random_%d" % n if ny == n and nz == n
            else "periodic_random_%dx%dx%d" % (n, ny, nz))
    return Case(name, n, ny, nz, 2 * np.pi, ly, Z_PERIODIC, lz, 0.0, re, 0.0,
                cfl, steps, u * s, v * s, w * s, np.zeros_like(u))


ENSEMBLE_SIZES = ((32, 32, 32), (64, 64, 64), (96, 96, 128), (128, 128, 192))


def case_ensemble(nboxes=64, seed=5, steps=100, sizes=ENSEMBLE_SIZES):
    """Ensemble of independent boxes of uneven sizes: sizes drawn uniformly
    from `sizes` (box-mix seed), box b seeded with 5000 + b.  Cubes of side
    32 or 64 are triply periodic 2 pi boxes with a Taylor-Green or a random
    solenoidal field (coin flip; the random one scaled to the Taylor-Green
    kinetic energy); the others are stretched channels (Poiseuille plus
    perturbation, RMS 0.1, |k| in [1, 8]).  Re log-uniform in [500, 4000],
    CFL 0.5."""
    rng = np.random.Generator(np.random.PCG64(seed))
    picks = rng.integers(0, len(sizes), nboxes)
    cases = []
    for b in range(nboxes):
        nx, ny, nz = sizes[int(picks[b])]
        brng = np.random.Generator(np.random.PCG64(5000 + b))
        re = float(np.exp(brng.uniform(np.log(500.0), np.log(4000.0))))
        if nx == ny == nz and nx <= 64:
            if brng.uniform() < 0.5:
                c = case_taylor_green(nx, steps=steps, re=re)
                c.cfl, c.dt = 0.5, 0.0
            else:
                c = case_periodic_random(nx, seed=5000 + b, re=re, steps=steps)
        else:
            c = case_channel(nx, ny, nz, re=re, steps=steps, seed=5000 + b)
        c.name = "box%02d_%s" % (b, c.name)
        cases.append(c)
    return cases


# ------------------------------------------------- immersed surface (IB) ----
def icosphere(level):
    """Unit sphere triangulated by `level` midpoint subdivisions of the
    icosahedron: (vertices (N x 3), triangles (F x 3), counter-clockwise seen
    from outside)."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
         (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    tris = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
            (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
            (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        mid = {}

        def midpoint(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                mid[key] = len(verts) - 1
            return mid[key]
        new = []
        for a, b, c in tris:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            new += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        tris = new
    return np.array(verts), np.array(tris, dtype=np.int64)


def ib_surface(center, radius, level, omega=(0.0, 0.0, 0.0), velocity=(0.0, 0.0, 0.0),
               two_sided=False):
    """Triangulated sphere standing in for a wet surface: markers at the face
    centroids, outward unit normals, face areas, the vertex list and the
    prescribed rigid motion of every marker (U = velocity + omega x (x -
    center)).  Returns a dict of numpy arrays."""
    unit, tris = icosphere(level)
    verts = np.asarray(center, dtype=np.float64) + radius * unit
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    xf = (a + b + c) / 3.0
    cr = np.cross(b - a, c - a)
    area = 0.5 * np.linalg.norm(cr, axis=1)
    nf = cr / (2.0 * area[:, None])
    rel = xf - np.asarray(center, dtype=np.float64)
    ub = np.asarray(velocity, dtype=np.float64)[None, :] + np.cross(
        np.asarray(omega, dtype=np.float64)[None, :], rel)
    return {"xf": xf, "nf": nf, "af": area, "tris": tris, "verts": verts, "ub": ub,
            "two_sided": np.full(len(tris), bool(two_sided))}
