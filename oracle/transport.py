"""Semi-Lagrangian transport with RK2 characteristics (Sec. 2.2) for the three models.

Test infrastructure only (see oracle/__init__.py).

Time: n_t cells of size h_t = 1/n_t (Sec. 2.2); states m_j = m(., j h_t), j = 0..n_t.
Space: positions in grid units xi = x/h; a stationary velocity v has shape (d, *n).

Readings (the paper only says "semi-Lagrangian, explicit RK2, unconditionally stable"):
* Characteristics (Heun's method, stationary v). Forward (state) departure points
      X*(x) = x - h_t v(x),  X-(x) = x - (h_t/2) (v(x) + I[v](X*(x)));
  backward (adjoint) departure points X+ are the same with v replaced by -v.
* Advection state (Eq. (1b)): m_{j+1} = I[m_j](X-).
* Advection adjoint (Eq. (4)), with mu = div v: along the characteristics of -v the
  adjoint obeys d lambda/d tau = lambda mu; Heun on that ODE gives
      Lam = I[lambda_{j+1}](X+),  S = I[lambda_{j+1} mu](X+),
      lambda_j = Lam + (h_t/2) (S + mu(x) (Lam + h_t S)).
  The product lambda_{j+1} mu is formed pointwise on the grid and interpolated once.
* Continuity state (Eq. (11b)): d pi/dt = -pi mu along the characteristics of v:
      P = I[pi_j](X-),  S = I[pi_j mu](X-),  pi~ = P - h_t S,
      pi_{j+1} = P - (h_t/2) (S + mu(x) pi~).
* Continuity adjoint: not printed in the paper; derived from the Lagrangian of
  problem (11) it is pure advection backward in time, lambda_j = I[lambda_{j+1}](X+).
"""
from __future__ import annotations

import numpy as np

from .interp import interp


def grid_index(n):
    """Grid positions in grid units, shape (d, *n)."""
    return np.stack(np.meshgrid(*[np.arange(ni, dtype=np.float64) for ni in n], indexing="ij"))


def departure_points_at(v, nt, sign, pts):
    """RK2 departure points (grid units) of the grid points pts (integer array (d, ...)).

    sign=+1 gives X- (state equation, characteristics of v);
    sign=-1 gives X+ (adjoint equation, characteristics of -v).
    """
    n = v.shape[1:]
    d = v.shape[0]
    ht = 1.0 / nt
    h = [2.0 * np.pi / ni for ni in n]
    pts = np.asarray(pts, dtype=np.int64)
    vp = np.stack([v[a][tuple(pts)] for a in range(d)])
    xstar = np.stack([pts[a] - sign * ht * vp[a] / h[a] for a in range(d)])
    vstar = np.stack([interp(v[a], xstar) for a in range(d)])
    return np.stack([pts[a] - sign * 0.5 * ht * (vp[a] + vstar[a]) / h[a] for a in range(d)])


def departure_points(v, nt, sign):
    """RK2 departure points in grid units at every grid point (see departure_points_at)."""
    return departure_points_at(v, nt, sign, grid_index(v.shape[1:]).astype(np.int64))


def state_step_at(model, mj, mu, xm, pts, nt):
    """m_{j+1} at the grid points pts from m_j, given their departure points xm = X-(pts)."""
    ht = 1.0 / nt
    p = interp(mj, xm)
    if model != "continuity":
        return p
    s = interp(mj * mu, xm)
    mup = mu[tuple(np.asarray(pts, dtype=np.int64))]
    return p - 0.5 * ht * (s + mup * (p - ht * s))


def adjoint_step_at(model, ln, mu, xp, pts, nt):
    """lambda_j at the grid points pts from lambda_{j+1}, given their departure points xp = X+(pts)."""
    ht = 1.0 / nt
    big = interp(ln, xp)
    if model == "continuity":
        return big
    s = interp(ln * mu, xp)
    mup = mu[tuple(np.asarray(pts, dtype=np.int64))]
    return big + 0.5 * ht * (s + mup * (big + ht * s))


def forward_states(model, m0, v, nt, mu=None, xm=None):
    """All states m_0..m_{n_t} of the state equation (advection or continuity)."""
    if xm is None:
        xm = departure_points(v, nt, +1)
    pts = grid_index(np.shape(m0)).astype(np.int64)
    states = [np.array(m0, dtype=np.float64)]
    for _ in range(nt):
        states.append(state_step_at(model, states[-1], mu, xm, pts, nt))
    return states


def adjoint_states(model, lam1, v, nt, mu=None, xp=None):
    """All adjoint states lambda_0..lambda_{n_t} given the terminal value lambda_{n_t} = lam1."""
    if xp is None:
        xp = departure_points(v, nt, -1)
    pts = grid_index(np.shape(lam1)).astype(np.int64)
    lams = [None] * (nt + 1)
    lams[nt] = np.array(lam1, dtype=np.float64)
    for j in range(nt - 1, -1, -1):
        lams[j] = adjoint_step_at(model, lams[j + 1], mu, xp, pts, nt)
    return lams
