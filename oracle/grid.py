"""Staggered Cartesian mesh of the fluid solver (Sec. 2.1: central second-order
finite differences on a staggered mesh; x, y periodic and z wall-normal with
no-slip, Sec. 4 and Sec. 5).  Test infrastructure only (see package header).

Storage of every field is ``a[k, j, i]`` (z slowest, x fastest).

Staggering (marker-and-cell):
    u at (x_i,      y_{j+1/2}, zc_k)   x-faces
    v at (x_{i+1/2}, y_j,      zc_k)   y-faces
    w at (x_{i+1/2}, y_{j+1/2}, z_k)   z-faces; with walls w[0] is the bottom
                                       wall (always 0) and the top wall face
                                       z_nz is not stored (also 0)
    p at (x_{i+1/2}, y_{j+1/2}, zc_k)   cell centres

x_i = i*dx, y_j = j*dy with dx = lx/nx, dy = ly/ny.  z faces z_0..z_nz; cell
widths dz_k = z_{k+1}-z_k; centres zc_k = (z_k+z_{k+1})/2; centre-to-centre
distances hc_k = zc_k - zc_{k-1} for k = 1..nz-1.  With walls hc_0 = dz_0/2 and
hc_nz = dz_{nz-1}/2 (wall to first/last centre); with periodic z the grid is
uniform and hc wraps.

The paper gives no stretching law.  The reading used here is the common tanh
clustering towards both walls: z_k = tanh(s(2k/nz-1))/tanh(s), s = stretch,
z in [-1, 1]; s = 0 gives a uniform mesh.
"""

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

Z_PERIODIC = 0
Z_WALLS = 1


@dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    zbc: int = Z_WALLS
    lz: float = 2.0          # periodic z only; walls always span [-1, 1]
    stretch: float = 0.0     # walls only: tanh clustering factor
    zfaces: Optional[np.ndarray] = None   # optional explicit nz+1 faces

    dx: float = field(init=False)
    dy: float = field(init=False)
    zf: np.ndarray = field(init=False)
    dz: np.ndarray = field(init=False)
    zc: np.ndarray = field(init=False)
    hc: np.ndarray = field(init=False)

    def __post_init__(self):
        self.dx = self.lx / self.nx
        self.dy = self.ly / self.ny
        nz = self.nz
        if self.zfaces is not None:
            zf = np.asarray(self.zfaces, dtype=np.float64).copy()
            assert zf.shape == (nz + 1,)
        elif self.zbc == Z_PERIODIC:
            zf = np.arange(nz + 1, dtype=np.float64) * (self.lz / nz)
        elif self.stretch > 0.0:
            s = self.stretch
            eta = 2.0 * np.arange(nz + 1, dtype=np.float64) / nz - 1.0
            zf = np.tanh(s * eta) / np.tanh(s)
        else:
            zf = -1.0 + 2.0 * np.arange(nz + 1, dtype=np.float64) / nz
        self.zf = zf
        self.dz = zf[1:] - zf[:-1]
        self.zc = 0.5 * (zf[1:] + zf[:-1])
        hc = np.empty(nz + 1)
        hc[1:nz] = self.zc[1:] - self.zc[:-1]
        if self.zbc == Z_WALLS:
            hc[0] = 0.5 * self.dz[0]
            hc[nz] = 0.5 * self.dz[nz - 1]
        else:
            hc[0] = 0.5 * (self.dz[nz - 1] + self.dz[0])
            hc[nz] = hc[0]
        self.hc = hc

    @property
    def walls(self) -> bool:
        return self.zbc == Z_WALLS

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    # coordinates of the staggered points (used by tests only)
    def x_face(self):
        return np.arange(self.nx) * self.dx

    def x_centre(self):
        return (np.arange(self.nx) + 0.5) * self.dx

    def y_face(self):
        return np.arange(self.ny) * self.dy

    def y_centre(self):
        return (np.arange(self.ny) + 0.5) * self.dy

    def cell_volume_uvp(self):
        """dx*dy*dz_k broadcast to [nz,1,1]: volume of u, v and p cells."""
        return (self.dx * self.dy * self.dz)[:, None, None]

    def cell_volume_w(self):
        """dx*dy*hc_k for the w faces k = 0..nz-1 (0 at the bottom wall)."""
        vol = self.dx * self.dy * self.hc[: self.nz].copy()
        if self.walls:
            vol[0] = 0.0
        return vol[:, None, None]
