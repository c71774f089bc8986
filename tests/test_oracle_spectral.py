"""Pins of the oracle's pseudo-spectral operators (Sec. 2.2) and Leray projector (Sec. 3.6)."""
import numpy as np
import pytest

from oracle import spectral as sp
from synth.inputs import random_fourier_field


def _grid(n):
    return np.meshgrid(*[2 * np.pi * np.arange(k) / k for k in n], indexing="ij")


@pytest.mark.parametrize("s", [1, 2, 3])
@pytest.mark.parametrize("n", [(16, 12), (8, 10, 12)])
def test_L_eigenfunctions(s, n):
    X = _grid(n)
    k = [1, -2, 3][: len(n)]
    phase = sum(kk * x for kk, x in zip(k, X))
    u = np.sin(phase + 0.2)
    lam = float(sum(kk * kk for kk in k)) ** s
    out = sp.apply_L(u[None], s)[0]
    np.testing.assert_allclose(out, lam * u, atol=1e-10 * lam)


def test_L_inverse_with_fixed_kernel():
    n = (12, 16)
    rng = np.random.default_rng(0)
    u = rng.standard_normal((2,) + n)
    alpha = 3e-2
    back = sp.apply_alphaL_inv(alpha * sp.apply_L(u, 2), 2, alpha)
    # the zero mode is annihilated by L and left at zero by the inverse
    np.testing.assert_allclose(back, u - u.mean(axis=(1, 2), keepdims=True), atol=1e-12)
    # zero mode of the inverse acts as 1/alpha (kernel entry set to one)
    const = np.ones((1,) + n)
    np.testing.assert_allclose(sp.apply_alphaL_inv(const, 2, alpha), const / alpha, rtol=1e-13)


def test_derivative_closed_form_and_nyquist_reading():
    n = (16, 8)
    X = _grid(n)
    f = np.sin(3 * X[0]) + np.cos(2 * X[1])
    g = sp.grad(f)
    np.testing.assert_allclose(g[0], 3 * np.cos(3 * X[0]), atol=1e-12)
    np.testing.assert_allclose(g[1], -2 * np.sin(2 * X[1]), atol=1e-12)
    # the Nyquist mode cos(n/2 x) has zero derivative under the k~ reading
    nyq = np.cos(8 * X[0])
    assert np.abs(sp.grad(nyq)).max() < 1e-12


def test_divergence_closed_form():
    n = (12, 12, 12)
    X = _grid(n)
    v = np.stack([np.sin(X[0]) * np.cos(X[1]), np.cos(2 * X[1]), np.sin(X[2] + X[0])])
    div = np.cos(X[0]) * np.cos(X[1]) - 2 * np.sin(2 * X[1]) + np.cos(X[2] + X[0])
    np.testing.assert_allclose(sp.div(v), div, atol=1e-12)


@pytest.mark.parametrize("n", [(16, 16), (8, 12, 10)])
def test_leray_projector_properties(n):
    rng = np.random.default_rng(1)
    d = len(n)
    u = rng.standard_normal((d,) + n)
    w = rng.standard_normal((d,) + n)
    pu = sp.leray(u)
    assert np.abs(sp.div(pu)).max() < 1e-12 * np.abs(u).max() * max(n)
    np.testing.assert_allclose(sp.leray(pu), pu, atol=1e-12)
    assert abs(sp.inner(pu, w, n) - sp.inner(u, sp.leray(w), n)) < 1e-11
    # gradients are annihilated, the mean is kept
    phi = random_fourier_field(n, 1, 3, rng)[0]
    assert np.abs(sp.leray(sp.grad(phi))).max() < 1e-12
    c = np.ones((d,) + n) * np.arange(1, d + 1).reshape((d,) + (1,) * d)
    np.testing.assert_allclose(sp.leray(c), c, atol=1e-13)


def test_regulariser_energy_closed_form():
    n = (16, 16)
    X = _grid(n)
    v = np.stack([np.sin(2 * X[0] + X[1]), np.zeros(n)])
    for s in (1, 2, 3):
        val = 0.5 * sp.inner(v, sp.apply_L(v, s), n)
        exact = 0.5 * 5.0 ** s * (2 * np.pi) ** 2 / 2
        assert abs(val - exact) < 1e-10 * exact


def test_line_derivative_closed_form_and_agreement_with_grad():
    """1D spectral derivative of a grid line: exact for trigonometric polynomials below Nyquist,
    zero for the Nyquist mode (reading of Sec. 2.2), and equal to the axis component of the 3D
    spectral gradient on every line of that axis."""
    L = 24
    x = 2 * np.pi * np.arange(L) / L
    np.testing.assert_allclose(sp.line_derivative(np.sin(3 * x) + 0.5 * np.cos(7 * x)),
                               3 * np.cos(3 * x) - 3.5 * np.sin(7 * x), atol=1e-12)
    np.testing.assert_allclose(sp.line_derivative(np.cos(L / 2 * x)), 0.0, atol=1e-12)
    f = np.random.default_rng(4).standard_normal((6, 10, 8))
    g = sp.grad(f)
    np.testing.assert_allclose(sp.line_derivative(np.moveaxis(f, 1, -1)), np.moveaxis(g[1], 1, -1), atol=1e-12)
    np.testing.assert_allclose(sp.line_derivative(np.moveaxis(f, 0, -1)), np.moveaxis(g[0], 0, -1), atol=1e-12)
