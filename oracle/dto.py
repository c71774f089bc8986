"""Discretise-then-optimise (exact discrete) gradient of the semi-Lagrangian objective.

Test infrastructure only (see oracle/__init__.py).

The paper optimises then discretises (Sec. 2.1): its adjoint is the discretised continuous adjoint,
so the reduced gradient differs from the derivative of the discrete objective by a discretisation
error. Here the discrete objective of the advection model (and of the incompressible model, whose
transport is advection with v kept in range(P)) is differentiated exactly:

    m_{j+1} = A m_j,  (A f)(x) = I[f](X-(x)),  J = 1/2 h^d sum (m_{n_t} - m_1)^2 + alpha/2 <v, L v>,
    X-_a(x) = x_a - (h_t / (2 h_a)) (v_a(x) + I[v_a](X*(x))),  X*_b(x) = x_b - h_t v_b(x) / h_b,

with positions in grid units. Backward: r_{n_t} = h^d (m_{n_t} - m_1), r_j = A^T r_{j+1}, and the
sensitivity of J to the departure points is G_a(x) = sum_{j<n_t} r_{j+1}(x) (d_a I[m_j])(X-(x)), where
d_a I[f](X) is the derivative of the cubic interpolant with respect to the a-th coordinate of the point
(grid units). The chain rule through the RK2 formula gives the Euclidean gradient with respect to the
grid values of v:

    dJ/dv_a(y) = -(h_t / (2 h_a)) [ G_a(y) + sum_x G_a(x) w(X*(x) -> y) ]
                 + (h_t^2 / (2 h_a)) sum_b (G_b(y) / h_b) (d_a I[v_b])(X*(y)),

and the L2 gradient is alpha L v + (1/h^d) dJ/dv (projected by P for the incompressible model).
"""
from __future__ import annotations

import itertools

import numpy as np

from . import spectral as sp
from .interp import _taps, cubic_lagrange_weights, interp, interp_transpose
from .transport import departure_points, grid_index


def cubic_lagrange_weight_derivatives(t):
    """d/dt of the Lagrange basis on nodes -1, 0, 1, 2 (see interp.cubic_lagrange_weights)."""
    return (
        -(3.0 * t * t - 6.0 * t + 2.0) / 6.0,
        (3.0 * t * t - 4.0 * t - 1.0) / 2.0,
        -(3.0 * t * t - 2.0 * t - 2.0) / 2.0,
        (3.0 * t * t - 1.0) / 6.0,
    )


def interp_grad(f, xi):
    """Gradient (d, ...) of the periodic cubic interpolant of f with respect to the point xi (grid
    units), inside each cell (the interpolant is only continuous across cell faces)."""
    d = f.ndim
    w, idx = _taps(f.shape, xi)
    t = xi - np.floor(xi)
    dw = [cubic_lagrange_weight_derivatives(t[a]) for a in range(d)]
    out = np.zeros((d,) + xi.shape[1:])
    for combo in itertools.product(range(4), repeat=d):
        val = f[tuple(idx[a][combo[a]] for a in range(d))]
        for a in range(d):
            wt = dw[a][combo[a]]
            for b in range(d):
                if b != a:
                    wt = wt * w[b][combo[b]]
            out[a] += wt * val
    return out


def _data_sensitivities(m0, m1, v, nt):
    """Forward states, departure points and G (see module docstring) for the advection transport."""
    n = m0.shape
    hd = sp.cell_volume(n)
    xm = departure_points(v, nt, +1)
    states = [np.array(m0, dtype=np.float64)]
    for _ in range(nt):
        states.append(interp(states[-1], xm))
    r = hd * (states[-1] - m1)
    G = np.zeros_like(v)
    for j in range(nt - 1, -1, -1):
        G += r[None] * interp_grad(states[j], xm)
        if j > 0:
            r = interp_transpose(r, xm, n)
    return states, G


def velocity_vjp(v, nt, G):
    """Euclidean gradient with respect to the grid values of v of sum_x G(x) . X-(x) (chain rule
    through the RK2 departure points)."""
    n = v.shape[1:]
    d = v.shape[0]
    ht = 1.0 / nt
    h = [2.0 * np.pi / ni for ni in n]
    base = grid_index(n)
    xstar = np.stack([base[a] - ht * v[a] / h[a] for a in range(d)])
    out = np.empty_like(v)
    for a in range(d):
        out[a] = -(ht / (2.0 * h[a])) * (G[a] + interp_transpose(G[a], xstar, n))
        acc = np.zeros(n)
        for b in range(d):
            acc += (G[b] / h[b]) * interp_grad(v[b], xstar)[a]
        out[a] += (ht * ht / (2.0 * h[a])) * acc
    return out


def objective(m0, m1, v, nt, s, alpha):
    """The discrete objective of the advection model (Eq. (1a) with the scheme of Sec. 2.2)."""
    n = m0.shape
    xm = departure_points(v, nt, +1)
    m = np.array(m0, dtype=np.float64)
    for _ in range(nt):
        m = interp(m, xm)
    return 0.5 * sp.cell_volume(n) * float(np.sum((m - m1) ** 2)) + 0.5 * alpha * sp.inner(v, sp.apply_L(v, s), n)


def gradient(m0, m1, v, nt, s, alpha, model="advection"):
    """L2 gradient of the discrete objective (advection; incompressible: projected by P)."""
    if model not in ("advection", "incompressible"):
        raise ValueError("the discrete gradient is built for the advection transport")
    n = m0.shape
    _, G = _data_sensitivities(m0, m1, v, nt)
    g = alpha * sp.apply_L(v, s) + velocity_vjp(v, nt, G) / sp.cell_volume(n)
    return sp.leray(g) if model == "incompressible" else g


def transport_vjp(m0, v, nt, gamma):
    """Exact Euclidean VJP of the transport map v -> m_{n_t} with cotangent gamma."""
    n = m0.shape
    xm = departure_points(v, nt, +1)
    states = [np.array(m0, dtype=np.float64)]
    for _ in range(nt):
        states.append(interp(states[-1], xm))
    r = np.array(gamma, dtype=np.float64)
    G = np.zeros_like(v)
    for j in range(nt - 1, -1, -1):
        G += r[None] * interp_grad(states[j], xm)
        if j > 0:
            r = interp_transpose(r, xm, n)
    return velocity_vjp(v, nt, G)
