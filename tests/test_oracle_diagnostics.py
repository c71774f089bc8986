"""Pins of the oracle's deformation diagnostics (the map y and det grad y shown with the results of
Sec. 3; for incompressible flows the paper reports det grad y = 1 to about 1e-13)."""
import numpy as np
import pytest

from oracle import spectral as sp
from oracle.diagnostics import deformation_displacement, det_from_displacement, det_grad_y
from oracle.interp import interp
from oracle.transport import forward_states, grid_index
from synth.inputs import smooth_velocity


def _x(n):
    return np.meshgrid(*[2 * np.pi * np.arange(k) / k for k in n], indexing="ij")


def _vel(n):
    """A compressible closed-form velocity, the same continuous field at every resolution."""
    x = _x(n)
    return np.stack([0.3 * np.sin(x[1]) * np.cos(x[0]) + 0.2, 0.25 * np.cos(2 * x[0]) + 0.1 * np.sin(x[1])])


def _img(n):
    x = _x(n)
    return np.sin(x[0]) * np.cos(2 * x[1]) + 0.5 * np.cos(x[0] + x[1])


def test_zero_velocity_gives_identity_map():
    n = (12, 10, 8)
    v = np.zeros((3,) + n)
    assert np.array_equal(deformation_displacement(v, 4), np.zeros((3,) + n))
    assert np.array_equal(det_grad_y(v, 4), np.ones(n))


def test_constant_velocity_is_a_rigid_shift():
    """y(x) = x - v for a constant v: u = -v/h in grid units after the unit time interval, and the
    map is volume preserving."""
    n = (16, 12)
    v = np.stack([np.full(n, 0.37), np.full(n, -1.1)])
    u = deformation_displacement(v, 5)
    h = [2 * np.pi / k for k in n]
    for a in range(2):
        np.testing.assert_allclose(u[a], -v[a] / h[a], rtol=0, atol=1e-12)
    np.testing.assert_allclose(det_grad_y(v, 5), 1.0, rtol=0, atol=1e-14)


def test_integer_shift_map_transports_the_image_exactly():
    """h_t v = 2 cells per step along axis 0: y is an exact shift by -2 n_t cells, and m0(y) equals
    the advected image (np.roll) exactly."""
    n = (16, 8)
    nt = 3
    h = 2 * np.pi / 16
    v = np.stack([np.full(n, 2.0 * h * nt), np.zeros(n)])
    u = deformation_displacement(v, nt)
    assert np.array_equal(u[0], np.full(n, -2.0 * nt))
    assert np.array_equal(u[1], np.zeros(n))
    m0 = np.random.default_rng(1).standard_normal(n)
    my = interp(m0, grid_index(n) + u)
    np.testing.assert_allclose(my, np.roll(m0, 2 * nt, axis=0), rtol=0, atol=1e-14)


def test_divergence_free_velocity_keeps_det_one():
    """Incompressible flow (Sec. 3.6): det grad y = 1 up to rounding."""
    rng = np.random.default_rng(3)
    v = sp.leray(smooth_velocity((24, 24, 24), 4, 2.0, rng, divergence_free=True))
    J = det_grad_y(v, 4)
    assert np.abs(J - 1.0).max() < 1e-12
    assert J.std() < 1e-13


def test_det_routes_agree_and_converge():
    """The continuity-equation route and det(I + grad(h u)) from the transported displacement are
    independent discretisations of the same quantity: their gap is small and shrinks at second order
    under refinement (n -> 2n, n_t -> 2 n_t)."""
    gaps = []
    for n, nt in (((32, 32), 4), ((64, 64), 8)):
        v = _vel(n)
        gaps.append(np.abs(det_grad_y(v, nt) - det_from_displacement(deformation_displacement(v, nt))).max())
    assert gaps[0] < 2e-3
    assert gaps[1] < gaps[0] / 3.0


def test_map_reproduces_the_advected_image():
    """m(., 1) = m0(y): the advection state solve and m0 interpolated at y agree to discretisation
    error, which shrinks under refinement (a wrong sign or orientation of u fails at once)."""
    errs = []
    for n, nt in (((32, 32), 4), ((64, 64), 8)):
        v = _vel(n)
        m0 = _img(n)
        mT = forward_states("advection", m0, v, nt)[-1]
        my = interp(m0, grid_index(n) + deformation_displacement(v, nt))
        errs.append(np.abs(mT - my).max())
    assert errs[0] < 5e-3
    assert errs[1] < errs[0] / 4.0


def test_mean_det_is_one_up_to_conservation_error():
    """A periodic diffeomorphism preserves total volume: mean(det grad y) -> 1 under refinement."""
    dev = []
    for n, nt in (((32, 32), 4), ((64, 64), 8)):
        dev.append(abs(det_grad_y(_vel(n), nt).mean() - 1.0))
    assert dev[0] < 1e-4
    assert dev[1] < dev[0] / 3.0


@pytest.mark.parametrize("bad", ["sign", "no_source"])
def test_pins_catch_planted_mistakes(bad):
    """The refinement pin fails for a displacement update with a flipped step sign or without the
    step displacement: the planted variants miss m0(y) = m(1) by O(1)."""
    n, nt = (32, 32), 4
    v = _vel(n)
    from oracle.transport import departure_points

    xm = departure_points(v, nt, +1)
    step = xm - grid_index(n)
    u = np.zeros_like(step)
    for _ in range(nt):
        u = np.stack([interp(u[a], xm) for a in range(2)]) + (-step if bad == "sign" else 0.0)
    m0 = _img(n)
    mT = forward_states("advection", m0, v, nt)[-1]
    assert np.abs(mT - interp(m0, grid_index(n) + u)).max() > 0.05
