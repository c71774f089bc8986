"""Objective, reduced gradient and preconditioner of the transport problems (Sec. 2.1-2.3).

Test infrastructure only (see oracle/__init__.py).

Discretisation (Sec. 2.2): L2 inner products are h^d-weighted sums; time integrals use the
trapezoidal rule with weights w_0 = w_{n_t} = 1/2, w_j = 1 otherwise.

Readings:
* Sign of the adjoint terminal value (Eq. (4)): the printed value -(m_1 - m(1)) together
  with g = alpha L v + int lambda grad m (Eq. (3)) gives the negative of the data gradient;
  the Lagrangian (Eq. (2)) as written gives lambda(1) = m_1 - m(1). The oracle uses
  lambda(1) = m_1 - m(1) with g = alpha L v + int_0^1 lambda grad m dt; a central
  finite-difference test of the discrete objective pins this sign.
* Continuity model (Sec. 3.7, problem (11)): adjoint -d_t lambda - v.grad lambda = 0,
  lambda(1) = pi_1 - pi(1); reduced gradient g = alpha L v - int_0^1 pi grad lambda dt.
* Incompressible model (Sec. 3.6): v is kept in range(P) (P the Leray projector);
  g = alpha L v + P b, and the preconditioned direction is s = -(alpha L)^{-1} P g.
  The forward/adjoint steps are those of the advection model (the source term with
  mu = div v is kept; it vanishes to roundoff on divergence-free v).
"""
from __future__ import annotations

import numpy as np

from . import spectral as sp
from .transport import adjoint_states, departure_points, forward_states

MODELS = ("advection", "continuity", "incompressible")


class Problem:
    """One registration problem: data m0, m1, n_t, model, regulariser order s, alpha."""

    def __init__(self, m0, m1, nt, model="advection", reg_order=2, alpha=1e-3):
        if model not in MODELS:
            raise ValueError(model)
        self.m0 = np.asarray(m0, dtype=np.float64)
        self.m1 = np.asarray(m1, dtype=np.float64)
        self.n = self.m0.shape
        self.d = self.m0.ndim
        self.nt = int(nt)
        self.model = model
        self.s = int(reg_order)
        self.alpha = float(alpha)
        self.hd = sp.cell_volume(self.n)
        self.counts = dict(obj=0, grad=0)

    # -- pieces -------------------------------------------------------------
    def reg_value(self, v):
        """alpha/2 <v, L v> (the regularisation term of Eq. (1a))."""
        return 0.5 * self.alpha * sp.inner(v, sp.apply_L(v, self.s), self.n)

    def mu(self, v):
        return sp.div(v)

    def states(self, v, xm=None, mu=None):
        if mu is None and self.model == "continuity":
            mu = self.mu(v)
        return forward_states("continuity" if self.model == "continuity" else "advection",
                              self.m0, v, self.nt, mu=mu, xm=xm)

    # -- objective / gradient / preconditioner --------------------------------
    def objective(self, v):
        """obj(v) = 1/2 ||m(1) - m_1||^2 + alpha/2 <v, L v> (Eq. (1a))."""
        self.counts["obj"] += 1
        mT = self.states(v)[-1]
        r = mT - self.m1
        return 0.5 * self.hd * float(np.sum(r * r)) + self.reg_value(v)

    def gradient(self, v, return_parts=False):
        """Reduced gradient (Eq. (3)) and objective at v; returns (g, obj)."""
        self.counts["grad"] += 1
        nt = self.nt
        ht = 1.0 / nt
        mu = self.mu(v)
        xm = departure_points(v, nt, +1)
        xp = departure_points(v, nt, -1)
        ms = self.states(v, xm=xm, mu=mu)
        r = ms[-1] - self.m1
        obj = 0.5 * self.hd * float(np.sum(r * r)) + self.reg_value(v)
        lam1 = self.m1 - ms[-1]
        adj_model = "continuity" if self.model == "continuity" else "advection"
        lams = adjoint_states(adj_model, lam1, v, nt, mu=mu, xp=xp)
        b = np.zeros_like(v)
        for j in range(nt + 1):
            wj = 0.5 if j in (0, nt) else 1.0
            if self.model == "continuity":
                b -= ht * wj * ms[j] * sp.grad(lams[j])
            else:
                b += ht * wj * lams[j] * sp.grad(ms[j])
        if self.model == "incompressible":
            b = sp.leray(b)
        g = self.alpha * sp.apply_L(v, self.s) + b
        if return_parts:
            return g, obj, dict(states=ms, adjoints=lams, body=b, mu=mu, xm=xm, xp=xp)
        return g, obj

    def precond(self, g):
        """s = -(alpha L)^{-1} g (Eq. (9) direction; P applied first for the incompressible model)."""
        if self.model == "incompressible":
            g = sp.leray(g)
        return -sp.apply_alphaL_inv(g, self.s, self.alpha)

    def inner(self, a, b):
        return sp.inner(a, b, self.n)
