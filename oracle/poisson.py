"""Pressure-increment Poisson solve of the fractional-step method (Sec. 2.1, the
elliptic equation that imposes mass conservation; Sec. 4 notes it is solved
with transposes across the x-y-periodic layout; FFTW3 is the FFT library).
Test infrastructure only (see package header).

Solves  D G phi = s  at the cell centres:
* discrete Fourier transform in x and y (numpy's FFT as a library step):
  the periodic second differences become -lambda_x - lambda_y with
  lambda_x = (2 - 2 cos(2 pi kx / nx)) / dx^2 (likewise y);
* per Fourier mode one tridiagonal system in z (Thomas; cyclic with
  Sherman-Morrison for periodic z):
      phi_{k-1}/(hc_k dz_k) + phi_{k+1}/(hc_{k+1} dz_k)
          - (1/(hc_k dz_k) + 1/(hc_{k+1} dz_k) + lambda_x + lambda_y) phi_k
      = s_k,
  with walls the wall fluxes are dropped (Neumann);
* gauge of the singular mode (kx, ky) = (0, 0): phi at k = 0 is pinned to 0
  and rows k = 1..nz-1 are solved (with periodic z the cyclic neighbours of
  k = 0 become this Dirichlet zero); row 0 then holds by compatibility of s.
  Finally the volume-weighted mean sum(phi dz_k) / sum(dz_k) is subtracted.
"""

import numpy as np

from .tridiag import thomas, cyclic_thomas


def z_poisson_coefficients(g):
    """(a, c, bz) of the z operator of D G: row k is
    a_k phi_{k-1} + bz_k phi_k + c_k phi_{k+1}."""
    nz = g.nz
    a = 1.0 / (g.hc[:nz] * g.dz)
    c = 1.0 / (g.hc[1:] * g.dz)
    if g.walls:
        a = a.copy()
        c = c.copy()
        a[0] = 0.0
        c[nz - 1] = 0.0
    bz = -(a + c)
    return a, c, bz


def modified_wavenumbers(n, h):
    """lambda_m = (2 - 2 cos(2 pi m / n)) / h^2, m = 0..n-1."""
    m = np.arange(n)
    return (2.0 - 2.0 * np.cos(2.0 * np.pi * m / n)) / h ** 2


def oracle_poisson(g, s):
    """phi with D G phi = s (s compatible: zero volume-weighted mean) and zero
    volume-weighted mean."""
    nz, ny, nx = g.shape
    a, c, bz = z_poisson_coefficients(g)
    lam = (modified_wavenumbers(nx, g.dx)[None, :]
           + modified_wavenumbers(ny, g.dy)[:, None])          # [ny, nx]
    s_hat = np.fft.fft2(s, axes=(1, 2))                         # [nz, ny, nx]

    b_full = bz[:, None, None] - lam[None, :, :]
    # the singular mode gets its own solve below; keep its row harmless here
    b_full = b_full.copy()
    b_full[:, 0, 0] = 1.0
    if g.walls:
        phi_hat = thomas(a, b_full, c, s_hat, axis=0)
    else:
        phi_hat = cyclic_thomas(a, b_full, c, s_hat, axis=0)

    # mode (0,0): phi_0 = 0, rows 1..nz-1 with phi_0 (and with periodic z the
    # cyclic neighbour phi_nz == phi_0) set to zero
    m0 = np.zeros(nz, dtype=complex)
    m0[1:] = thomas(a[1:], bz[1:], c[1:], s_hat[1:, 0, 0], axis=0)
    phi_hat[:, 0, 0] = m0

    phi = np.real(np.fft.ifft2(phi_hat, axes=(1, 2)))
    wmean = (phi * g.dz[:, None, None]).sum() / (g.dz.sum() * nx * ny)
    return phi - wmean
