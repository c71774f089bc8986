"""Pins of the oracle's periodic cubic Lagrange interpolation (semi-Lagrangian gather, Sec. 2.2)."""
import numpy as np
import pytest
from scipy.interpolate import BarycentricInterpolator

from oracle.interp import cubic_lagrange_weights, interp, interp_transpose


def test_weights_match_library_lagrange_polynomials():
    # Library routine: scipy's polynomial interpolant through nodes -1,0,1,2 for each basis vector.
    ts = np.linspace(-0.3, 1.3, 17)
    w = np.stack(cubic_lagrange_weights(ts))
    for j in range(4):
        e = np.zeros(4)
        e[j] = 1.0
        poly = BarycentricInterpolator(np.array([-1.0, 0.0, 1.0, 2.0]), e)
        np.testing.assert_allclose(w[j], poly(ts), atol=1e-13)


def test_weights_reproduce_monomials_up_to_cubic():
    t = np.random.default_rng(0).uniform(0, 1, 50)
    w = cubic_lagrange_weights(t)
    nodes = (-1.0, 0.0, 1.0, 2.0)
    for p in range(4):
        np.testing.assert_allclose(sum(wj * x ** p for wj, x in zip(w, nodes)), t ** p, atol=1e-14)


def test_integer_positions_are_exact():
    rng = np.random.default_rng(1)
    f = rng.standard_normal((7, 9, 5))
    xi = np.stack(np.meshgrid(*[np.arange(k, dtype=float) for k in f.shape], indexing="ij"))
    assert np.array_equal(interp(f, xi), f)
    # integer shifts (with wrap, negative too) are exact rolls
    shift = np.array([2.0, -3.0, 7.0]).reshape(3, 1, 1, 1)
    out = interp(f, xi + shift)
    assert np.array_equal(out, np.roll(f, (-2, 3, -7), axis=(0, 1, 2)))


def test_cubic_polynomials_reproduced_away_from_wrap():
    rng = np.random.default_rng(2)
    n = (20, 22, 18)
    xs = [np.arange(k, dtype=float) for k in n]
    X = np.meshgrid(*xs, indexing="ij")
    c = rng.standard_normal(6)
    f = (c[0] + c[1] * X[0] ** 3 + c[2] * X[1] ** 2 * X[2] + c[3] * X[0] * X[1] * X[2]
         + c[4] * X[2] ** 3 + c[5] * X[0] ** 2 * X[1])
    pts = np.stack([rng.uniform(2, k - 4, 200) for k in n])
    exact = (c[0] + c[1] * pts[0] ** 3 + c[2] * pts[1] ** 2 * pts[2] + c[3] * pts[0] * pts[1] * pts[2]
             + c[4] * pts[2] ** 3 + c[5] * pts[0] ** 2 * pts[1])
    np.testing.assert_allclose(interp(f, pts), exact, rtol=1e-11, atol=1e-9)


def test_smooth_interpolation_converges_fourth_order():
    errs = []
    rng = np.random.default_rng(3)
    pts01 = rng.uniform(0, 1, (2, 400))
    for N in (16, 32, 64):
        h = 2 * np.pi / N
        x = np.arange(N) * h
        X = np.meshgrid(x, x, indexing="ij")
        f = np.sin(X[0] + 0.3) * np.cos(2 * X[1])
        P = pts01 * 2 * np.pi
        exact = np.sin(P[0] + 0.3) * np.cos(2 * P[1])
        errs.append(np.abs(interp(f, P / h) - exact).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.6), (errs, rates)


def test_transpose_dot_product():
    rng = np.random.default_rng(4)
    n = (9, 10, 11)
    a = rng.standard_normal(n)
    xi = np.stack([rng.uniform(-20, 20, (6, 7)) for _ in n])
    r = rng.standard_normal((6, 7))
    lhs = float(np.sum(interp(a, xi) * r))
    rhs = float(np.sum(a * interp_transpose(r, xi, n)))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)
