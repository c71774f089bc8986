"""Periodic tensor-product cubic Lagrange interpolation (the semi-Lagrangian gather, Sec. 2.2).

Test infrastructure only (see oracle/__init__.py).

Reading: the paper defers the interpolation order to its cited works; the library uses
tensor-product 4-point cubic Lagrange interpolation on nodes {-1, 0, 1, 2}, periodic
wrap, no prefilter. In grid units xi = X/h, i0 = floor(xi), t = xi - i0 and the
weights are the Lagrange basis polynomials through t in {-1, 0, 1, 2}:
    w_-1 = -t(t-1)(t-2)/6,  w_0 = (t+1)(t-1)(t-2)/2,
    w_1  = -(t+1)t(t-2)/2,  w_2 = (t+1)t(t-1)/6.
"""
from __future__ import annotations

import itertools

import numpy as np


def cubic_lagrange_weights(t):
    """Lagrange basis on nodes -1, 0, 1, 2 evaluated at t (array); returns 4 arrays."""
    return (
        -t * (t - 1.0) * (t - 2.0) / 6.0,
        (t + 1.0) * (t - 1.0) * (t - 2.0) / 2.0,
        -(t + 1.0) * t * (t - 2.0) / 2.0,
        (t + 1.0) * t * (t - 1.0) / 6.0,
    )


def _taps(f_shape, xi):
    d = len(f_shape)
    i0 = np.floor(xi).astype(np.int64)
    t = xi - i0
    w = [cubic_lagrange_weights(t[a]) for a in range(d)]
    idx = [[(i0[a] + o) % f_shape[a] for o in (-1, 0, 1, 2)] for a in range(d)]
    return w, idx


def interp(f, xi):
    """Values of the periodic cubic interpolant of grid field f at points xi.

    f: array of shape n (d axes); xi: array (d, ...) of positions in grid units
    (axis a coordinate divided by h_a). Returns an array of shape xi.shape[1:].
    """
    d = f.ndim
    w, idx = _taps(f.shape, xi)
    out = np.zeros(xi.shape[1:])
    for combo in itertools.product(range(4), repeat=d):
        wt = w[0][combo[0]]
        for a in range(1, d):
            wt = wt * w[a][combo[a]]
        out += wt * f[tuple(idx[a][combo[a]] for a in range(d))]
    return out


def interp_transpose(r, xi, n):
    """Exact transpose of interp(., xi): scatters r (shape xi.shape[1:]) onto a grid of shape n."""
    d = len(n)
    w, idx = _taps(n, xi)
    out = np.zeros(n)
    for combo in itertools.product(range(4), repeat=d):
        wt = w[0][combo[0]]
        for a in range(1, d):
            wt = wt * w[a][combo[a]]
        np.add.at(out, tuple(idx[a][combo[a]] for a in range(d)), wt * r)
    return out
