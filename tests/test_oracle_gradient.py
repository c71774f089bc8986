"""Pins of the oracle's objective, reduced gradient and preconditioner (Eqs. (1a), (3), (4), (9)).

The gradient is optimize-then-discretize (Sec. 2.1), so it is not the exact derivative of the
discrete objective: the central finite-difference check agrees only to discretisation error,
and the pin is that this error falls under refinement (N -> 2N, n_t -> 2 n_t). A wrong sign of
the adjoint terminal value, a dropped time-quadrature weight or a transposed component would
leave an O(1) mismatch that does not fall.
"""
import numpy as np
import pytest

from oracle import spectral as sp
from oracle.problem import Problem


def _fields(n, model):
    X = np.meshgrid(*[2 * np.pi * np.arange(k) / k for k in n], indexing="ij")
    d = len(n)
    m0 = 0.5 + 0.2 * np.sin(X[0]) * np.cos(2 * X[1]) + 0.1 * np.cos(X[-1] + 0.3)
    m1 = 0.5 + 0.2 * np.sin(X[0] + 0.2) * np.cos(2 * X[1] - 0.1) + 0.1 * np.cos(X[-1] + 0.5)
    v = np.stack([0.15 * np.sin(X[(a + 1) % d] + a) + 0.1 * np.cos(2 * X[a]) for a in range(d)])
    dv = np.stack([np.cos(X[(a + 2) % d] + 0.5 * a) * np.sin(X[a]) for a in range(d)])
    if model == "continuity":
        m0, m1 = m0 + 0.5, m1 + 0.5
    if model == "incompressible":
        v, dv = sp.leray(v), sp.leray(dv)
    return m0, m1, v, dv


@pytest.mark.parametrize("model", ["advection", "continuity", "incompressible"])
@pytest.mark.parametrize("d", [2, 3])
def test_gradient_matches_central_fd_to_vanishing_discretisation_error(model, d):
    sizes = [(16, 2), (32, 4), (64, 8)] if d == 2 else [(12, 2), (24, 4)]
    errs = []
    for N, nt in sizes:
        n = (N,) * d
        m0, m1, v, dv = _fields(n, model)
        P = Problem(m0, m1, nt=nt, model=model, reg_order=2 if model == "advection" else 1, alpha=1e-3)
        g, J = P.gradient(v)
        eps = 1e-4
        fd = (P.objective(v + eps * dv) - P.objective(v - eps * dv)) / (2 * eps)
        an = P.inner(g, dv)
        errs.append(abs(fd - an) / abs(fd))
    assert errs[-1] < 0.05, errs
    for a, b in zip(errs[:-1], errs[1:]):
        assert b < a / 2.0, errs


def test_regularisation_gradient_is_exact():
    # With m1 = m(1) the data term vanishes at first order: g = alpha L v + (terms ~ residual);
    # at v = 0 and m1 = m0 the gradient is exactly zero.
    n = (12, 12)
    m0 = np.random.default_rng(0).standard_normal(n)
    P = Problem(m0, m0.copy(), nt=4, model="advection", reg_order=2, alpha=1e-2)
    g, J = P.gradient(np.zeros((2,) + n))
    assert J == 0.0 and np.abs(g).max() == 0.0
    # with the data term switched off (m1 = transported m0) the objective is the regulariser
    X = np.meshgrid(*[2 * np.pi * np.arange(k) / k for k in n], indexing="ij")
    v = np.stack([0.1 * np.sin(X[1]), 0.2 * np.cos(X[0])])
    P2 = Problem(m0, m0, nt=4, model="advection", reg_order=1, alpha=1e-2)
    m1 = P2.states(v)[-1]
    P3 = Problem(m0, m1, nt=4, model="advection", reg_order=1, alpha=1e-2)
    g3, J3 = P3.gradient(v)
    np.testing.assert_allclose(g3, 1e-2 * sp.apply_L(v, 1), atol=1e-15)
    exact = 0.5 * 1e-2 * (0.01 + 0.04) * (2 * np.pi) ** 2 / 2
    assert abs(J3 - exact) < 1e-12


@pytest.mark.parametrize("model", ["advection", "continuity", "incompressible"])
def test_preconditioner_inverts_regulariser(model):
    n = (16, 16)
    rng = np.random.default_rng(2)
    P = Problem(np.zeros(n), np.zeros(n), nt=2, model=model, reg_order=2, alpha=5e-3)
    v = rng.standard_normal((2,) + n)
    if model == "incompressible":
        v = sp.leray(v)
    v -= v.mean(axis=(1, 2), keepdims=True)
    s = P.precond(5e-3 * sp.apply_L(v, 2))
    np.testing.assert_allclose(s, -v, atol=1e-11)
    if model == "incompressible":
        g = rng.standard_normal((2,) + n)
        assert np.abs(sp.div(P.precond(g))).max() < 1e-10


def test_descent_direction():
    n = (16, 16)
    rng = np.random.default_rng(3)
    X = np.meshgrid(*[2 * np.pi * np.arange(k) / k for k in n], indexing="ij")
    m0 = np.sin(X[0]) * np.cos(X[1])
    m1 = np.sin(X[0] - 0.3) * np.cos(X[1] + 0.2)
    P = Problem(m0, m1, nt=4, model="advection", reg_order=2, alpha=1e-3)
    v = np.zeros((2,) + n)
    g, J = P.gradient(v)
    s = P.precond(g)
    assert P.inner(g, s) < 0
    assert P.objective(v + 1e-3 * s) < J
