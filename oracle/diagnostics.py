"""Deformation diagnostics of a stationary velocity: the map y and det grad y.

Test infrastructure only (see oracle/__init__.py).

The paper shows, with its results, the computed map y and the determinant of its deformation
gradient (Fig. 3 and the incompressible results of Sec. 3.6, where det grad y equals 1 to about
1e-13), but does not print how either is computed. Readings:

* y maps a grid point at t = 1 back to the origin of its characteristic at t = 0, so that the
  transported image is m(x, 1) = m_0(y(x)) (advection model, Eq. (1b)). Write y = x + h u with a
  periodic displacement u in grid units. The semi-Lagrangian step m_{j+1} = I[m_j](X-) composes
  y_{j+1}(x) = y_j(X-(x)), which for the displacement reads
      u_0 = 0,   u_{j+1} = I[u_j](X-) + (X- - x)        (X- in grid units, Sec. 2.2).
* det grad y is the Jacobian determinant of the inverse flow map. It is the density of the
  transported uniform measure, so it solves the continuity equation (Eq. (11b)) with initial
  value 1: d_t J + div(J v) = 0, J(0) = 1, det grad y = J(1). It is computed with the continuity
  state scheme of the transport module from pi_0 = 1. For div v = 0 the scheme keeps J = 1 up to
  rounding, which is the behaviour the paper reports for incompressible flows.

A second, independent route to det grad y differentiates the displacement spectrally,
det(I + grad(h u)); the two agree to discretisation error (a test cross-check, not the reading).
"""
from __future__ import annotations

import numpy as np

from .interp import interp
from .spectral import div, grad
from .transport import departure_points, forward_states, grid_index


def deformation_displacement(v, nt):
    """Displacement u (grid units, shape (d, *n)) of the map y = x + h u after n_t steps."""
    xm = departure_points(v, nt, +1)
    step = xm - grid_index(v.shape[1:])  # X- - x, the departure displacement of one step
    u = np.zeros_like(step)
    for _ in range(nt):
        u = np.stack([interp(u[a], xm) for a in range(u.shape[0])]) + step
    return u


def det_grad_y(v, nt):
    """det grad y as the continuity state at t = 1 started from the constant 1."""
    n = v.shape[1:]
    return forward_states("continuity", np.ones(n), v, nt, mu=div(v))[-1]


def det_from_displacement(u):
    """det(I + grad(h u)) with spectral first derivatives (cross-check route)."""
    n = u.shape[1:]
    d = u.shape[0]
    h = [2.0 * np.pi / ni for ni in n]
    jac = np.empty((d, d) + tuple(n))
    for a in range(d):
        ga = grad(h[a] * u[a])
        for b in range(d):
            jac[a, b] = ga[b] + (1.0 if a == b else 0.0)
    return np.linalg.det(np.moveaxis(jac, (0, 1), (-2, -1)))
