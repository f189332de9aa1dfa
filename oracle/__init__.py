"""FP64 CPU oracle for one fractional step of the staggered-grid Navier-Stokes
integrator of the FSEI solver (arXiv 2103.15187, Sec. 2.1 and Sec. 3.1).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA library (no kernels, headers, helpers, tables or constants); the two meet
only through the seeded input generators, which hold none of the method's
arithmetic.

The oracle is plain, slow numpy in float64, written to be checked against the
paper by eye:

* ``grid``      -- staggered mesh, z stretching and z metrics
* ``operators`` -- advection H, viscous L, gradient G, divergence D (Sec. 2.1)
* ``tridiag``   -- Thomas algorithm and its cyclic (Sherman-Morrison) variant
                   (Sec. 3.1)
* ``poisson``   -- pressure-increment Poisson solve, FFT in x, y + tridiagonal
                   in z, with the gauge of the singular mode
* ``step``      -- one AB2 / Crank-Nicolson fractional step (Eq. 3) and its
                   third-order Runge-Kutta variant
* ``adjoint``   -- the exact transpose of that step (discrete adjoint)
* ``rheology``  -- the Carreau-Yasuda (shear-thinning) stress, as an explicit
                   remainder beside the implicit Newtonian viscous term
* ``ib``        -- immersed-boundary forcing by moving least squares and the
                   hydrodynamic loads on the immersed surface (Eqs. 4-7)

Pins (tests/test_oracle_*.py) tie every function to something other than
itself: dense direct solves, closed-form single-mode amplification factors,
discrete divergence after projection, kinetic-energy conservation of the
advection operator, a discrete Poiseuille steady state, manufactured-solution
convergence order and the adjoint dot-product identity.
"""

from .grid import Grid  # noqa: F401
from .step import oracle_step, oracle_step_rk3, oracle_cfl_dt, oracle_stats  # noqa: F401
from .poisson import oracle_poisson  # noqa: F401
