"""Pins of the oracle's tridiagonal solvers (Sec. 3.1: Thomas' algorithm, with a
Sherman-Morrison perturbation for the periodic directions) against a dense
LAPACK solve of the assembled matrix."""

import numpy as np
import pytest

from oracle.tridiag import thomas, cyclic_thomas

pytestmark = pytest.mark.filterwarnings("error")


def _dense(a, b, c, cyclic):
    n = len(b)
    m = np.zeros((n, n), dtype=np.result_type(a, b, c))
    for i in range(n):
        m[i, i] = b[i]
        if i > 0:
            m[i, i - 1] = a[i]
        if i < n - 1:
            m[i, i + 1] = c[i]
    if cyclic:
        m[0, n - 1] = a[0]
        m[n - 1, 0] = c[n - 1]
    return m


@pytest.mark.parametrize("n", [3, 5, 17, 64])
def test_thomas_matches_dense_solve(n):
    rng = np.random.default_rng(n)
    a = rng.uniform(-1, 1, n)
    c = rng.uniform(-1, 1, n)
    b = np.abs(a) + np.abs(c) + rng.uniform(0.1, 1.0, n)
    d = rng.standard_normal((n, 4, 3))
    x = thomas(a, b, c, d, axis=0)
    m = _dense(a, b, c, False)
    ref = np.linalg.solve(m, d.reshape(n, -1)).reshape(d.shape)
    assert np.max(np.abs(x - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("n", [3, 4, 9, 32, 96])
def test_cyclic_thomas_matches_dense_solve(n):
    rng = np.random.default_rng(100 + n)
    a = rng.uniform(-1, 1, n)
    c = rng.uniform(-1, 1, n)
    b = np.abs(a) + np.abs(c) + rng.uniform(0.1, 1.0, n)
    d = rng.standard_normal((5, n))
    x = cyclic_thomas(a, b, c, d, axis=1)
    m = _dense(a, b, c, True)
    ref = np.linalg.solve(m, d.T).T
    assert np.max(np.abs(x - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_per_line_coefficients_and_complex_rhs():
    """One matrix per line (the Poisson z-systems have a mode-dependent
    diagonal) and complex right-hand sides."""
    rng = np.random.default_rng(7)
    n, lines = 12, 6
    a = rng.uniform(-1, 1, (n, lines))
    c = rng.uniform(-1, 1, (n, lines))
    b = np.abs(a) + np.abs(c) + 0.5
    d = rng.standard_normal((n, lines)) + 1j * rng.standard_normal((n, lines))
    x = thomas(a, b, c, d, axis=0)
    xc = cyclic_thomas(a, b, c, d, axis=0)
    for l in range(lines):
        ref = np.linalg.solve(_dense(a[:, l], b[:, l], c[:, l], False), d[:, l])
        refc = np.linalg.solve(_dense(a[:, l], b[:, l], c[:, l], True), d[:, l])
        assert np.max(np.abs(x[:, l] - ref)) <= 1e-13 * np.max(np.abs(ref))
        assert np.max(np.abs(xc[:, l] - refc)) <= 1e-13 * np.max(np.abs(refc))
