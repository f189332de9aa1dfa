"""Tridiagonal solvers of the approximately factorised implicit step (Sec. 3.1:
one tridiagonal matrix per direction, inverted with Thomas' algorithm, with a
Sherman-Morrison perturbation in the two periodic directions).  Test
infrastructure only (see package header).

Row i of the system reads  a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i.
All lines along ``axis`` are solved at once (numpy vectorisation over the
other axes).  a, b and c are either 1-D arrays of the line length (one matrix
for every line) or full arrays shaped like d (one matrix per line).
"""

import numpy as np


def _coef_front(coef, axis, d_front_shape):
    """Coefficient array with the solve axis first, broadcast to d's shape."""
    coef = np.asarray(coef)
    if coef.ndim == 1:
        coef = coef.reshape((-1,) + (1,) * (len(d_front_shape) - 1))
    else:
        coef = np.moveaxis(coef, axis, 0)
    return np.broadcast_to(coef, d_front_shape)


def thomas(a, b, c, d, axis=0):
    """Thomas' algorithm (Gaussian elimination without pivoting of a
    tridiagonal matrix).  a[0] and c[n-1] are ignored."""
    dd = np.moveaxis(np.asarray(d), axis, 0)
    shape = dd.shape
    a = _coef_front(a, axis, shape)
    b = _coef_front(b, axis, shape)
    c = _coef_front(c, axis, shape)
    n = shape[0]
    dtype = np.result_type(dd.dtype, b.dtype, np.float64)
    cp = np.empty(shape, dtype=dtype)
    dp = np.empty(shape, dtype=dtype)
    # forward elimination
    cp[0] = c[0] / b[0]
    dp[0] = dd[0] / b[0]
    for i in range(1, n):
        den = b[i] - a[i] * cp[i - 1]
        cp[i] = c[i] / den
        dp[i] = (dd[i] - a[i] * dp[i - 1]) / den
    # back substitution
    x = np.empty(shape, dtype=dtype)
    x[n - 1] = dp[n - 1]
    for i in range(n - 2, -1, -1):
        x[i] = dp[i] - cp[i] * x[i + 1]
    return np.moveaxis(x, 0, axis)


def cyclic_thomas(a, b, c, d, axis=0):
    """Periodic tridiagonal system: a_0 couples x_{n-1} into row 0 and c_{n-1}
    couples x_0 into row n-1.

    Sherman-Morrison: A = T + u v^T with u = (g, 0, ..., 0, c_{n-1}),
    v = (1, 0, ..., 0, a_0/g), g = -b_0.  T is A without its two corner
    entries and with its first and last diagonal entries changed to b_0 - g
    and b_{n-1} - c_{n-1} a_0 / g.  Then x = y - (v.y / (1 + v.z)) z with
    T y = d and T z = u, both by Thomas' algorithm.
    """
    dd = np.moveaxis(np.asarray(d), axis, 0)
    shape = dd.shape
    n = shape[0]
    assert n >= 3
    a = _coef_front(a, axis, shape)
    c = _coef_front(c, axis, shape)
    b = np.array(_coef_front(b, axis, shape),
                 dtype=np.result_type(np.asarray(b).dtype, np.float64))
    gam = -b[0].copy()
    a0 = a[0]
    cn = c[n - 1]
    b[0] = b[0] - gam
    b[n - 1] = b[n - 1] - cn * a0 / gam
    uvec = np.zeros(shape, dtype=b.dtype)
    uvec[0] = gam
    uvec[n - 1] = cn
    y = thomas(a, b, c, dd, axis=0)
    z = thomas(a, b, c, uvec, axis=0)
    vy = y[0] + (a0 / gam) * y[n - 1]
    vz = z[0] + (a0 / gam) * z[n - 1]
    x = y - (vy / (1.0 + vz)) * z
    return np.moveaxis(x, 0, axis)
