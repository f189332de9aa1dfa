"""Pins of the oracle's discrete adjoint: every transposed piece satisfies the
dot-product identity <A x, y> = <x, A^T y> against its forward operator, and
the whole adjoint step satisfies it against the step's linearisation.  The
step is quadratic in u^n and linear in p^n, H^{n-1} and f, so the central
difference [F(x + e d) - F(x - e d)] / (2e) is its exact directional
derivative (up to rounding) -- an independent reference for J d."""

import numpy as np
import pytest

from oracle.grid import Grid, Z_PERIODIC, Z_WALLS
from oracle import operators as op
from oracle import adjoint as adj
from oracle import step as st
from oracle.poisson import oracle_poisson

GRIDS = [
    Grid(8, 8, 8, 2 * np.pi, 2 * np.pi, Z_PERIODIC, lz=2 * np.pi),
    Grid(12, 10, 9, 2.0, 1.5, Z_WALLS, stretch=2.0),
    Grid(8, 6, 10, 1.0, 2.0, Z_PERIODIC, lz=1.3),
]
IDS = ["periodic8", "walls12x10x9", "periodic8x6x10"]


def _r(g, seed, n=3):
    rng = np.random.default_rng(seed)
    out = [rng.standard_normal(g.shape) for _ in range(n)]
    if g.walls and n >= 3:
        out[2][0] = 0.0
    return out


def _dot(xs, ys):
    return sum(float((x * y).sum()) for x, y in zip(xs, ys))


def _close(a, b, tol=1e-12):
    assert abs(a - b) <= tol * max(abs(a), abs(b), 1e-300), (a, b)


@pytest.mark.parametrize("g", GRIDS, ids=IDS)
def test_gradient_divergence_transposes(g):
    p = _r(g, 1, 1)[0]
    y = _r(g, 2)
    _close(_dot(op.gradient(g, p), y), _dot([p], [adj.gradient_T(g, *y)]))
    x = _r(g, 3)
    s = _r(g, 4, 1)[0]
    _close(_dot([op.divergence(g, *x)], [s]), _dot(x, adj.divergence_T(g, s)))


@pytest.mark.parametrize("g", GRIDS, ids=IDS)
def test_viscous_and_poisson_operator_transposes(g):
    x, y = _r(g, 5), _r(g, 6)
    _close(_dot(op.viscous(g, *x), y), _dot(x, adj.viscous_T(g, *y)))
    a, b = _r(g, 7, 1)[0], _r(g, 8, 1)[0]
    _close(_dot([op.laplacian_p(g, a)], [b]), _dot([a], [adj.laplacian_p_T(g, b)]))


@pytest.mark.parametrize("g", GRIDS, ids=IDS)
def test_sweep_transposes(g):
    beta = 3e-3
    x, y = _r(g, 9), _r(g, 10)
    fwd = (st.sweep_z_centre(g, beta, st.sweep_y(g, beta, st.sweep_x(g, beta, x[0]))),
           st.sweep_z_centre(g, beta, st.sweep_y(g, beta, st.sweep_x(g, beta, x[1]))),
           st.sweep_z_face(g, beta, st.sweep_y(g, beta, st.sweep_x(g, beta, x[2]))))
    _close(_dot(fwd, y), _dot(x, adj.sweeps_T(g, beta, *y)))


@pytest.mark.parametrize("g", GRIDS, ids=IDS)
def test_projection_poisson_transpose(g):
    """phi = P(D u) restricted to divergences: <P D x, y> = <x, D^T P^T y>."""
    x = _r(g, 11)
    y = _r(g, 12, 1)[0]
    lhs = float((oracle_poisson(g, op.divergence(g, *x)) * y).sum())
    rhs = _dot(x, adj.divergence_T(g, adj.poisson_T(g, y)))
    _close(lhs, rhs, 1e-11)


@pytest.mark.parametrize("g", GRIDS, ids=IDS)
def test_advection_jacobian_transpose(g):
    u = _r(g, 13)
    d = _r(g, 14)
    y = _r(g, 15)
    eps = 1e-3
    plus = op.advection(g, *[a + eps * b for a, b in zip(u, d)])
    minus = op.advection(g, *[a - eps * b for a, b in zip(u, d)])
    jd = [(p - m) / (2 * eps) for p, m in zip(plus, minus)]
    _close(_dot(jd, y), _dot(d, adj.advection_T(g, *u, *y)), 1e-11)


def _step_out(g, s, f, prm):
    new, _ = st.oracle_step(g, s, f, **prm)
    return [new[k] for k in ("u", "v", "w", "p", "hu", "hv", "hw")]


@pytest.mark.parametrize("g", GRIDS, ids=IDS)
@pytest.mark.parametrize("have_prev", [0, 1])
def test_adjoint_step_dot_product(g, have_prev):
    """<J d, y> = <d, J^T y> for the full step, d over (u, v, w, p, H, f)."""
    rng = np.random.default_rng(20 + have_prev)
    base = _r(g, 16) + _r(g, 17, 1) + _r(g, 18)
    f = _r(g, 19)
    dirs = _r(g, 21) + _r(g, 22, 1) + _r(g, 23)
    df = _r(g, 24)
    cot = _r(g, 25) + _r(g, 26, 1) + _r(g, 27)
    prm = dict(re=70.0, dt=5e-3, cfl=0.0)
    keys = ("u", "v", "w", "p", "hu", "hv", "hw")
    eps = 1e-4

    def state(sign):
        s = {k: base[i] + sign * eps * dirs[i] for i, k in enumerate(keys)}
        s["have_prev_h"] = have_prev
        return s, tuple(a + sign * eps * b for a, b in zip(f, df))

    sp, fp = state(1)
    sm, fm = state(-1)
    out_p = _step_out(g, sp, fp, prm)
    out_m = _step_out(g, sm, fm, prm)
    jd = [(a - b) / (2 * eps) for a, b in zip(out_p, out_m)]
    s0 = {k: base[i] for i, k in enumerate(keys)}
    s0["have_prev_h"] = have_prev
    cd = {k: cot[i] for i, k in enumerate(keys)}
    res = adj.oracle_adjoint_step(g, s0, cd, f, re=prm["re"], dt=prm["dt"])
    lhs = _dot(jd, cot)
    rhs = _dot(dirs, [res[k] for k in keys]) + _dot(df, [res["fx"], res["fy"], res["fz"]])
    del rng
    _close(lhs, rhs, 1e-9)
