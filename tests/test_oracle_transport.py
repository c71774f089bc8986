"""Pins of the oracle's semi-Lagrangian transport (Sec. 2.2; Eqs. (1b), (4), (11b))."""
import numpy as np
import pytest

from oracle import spectral as sp
from oracle.transport import adjoint_states, departure_points, forward_states, grid_index
from synth.inputs import random_fourier_field


def _grid(n):
    return np.meshgrid(*[2 * np.pi * np.arange(k) / k for k in n], indexing="ij")


@pytest.mark.parametrize("model", ["advection", "continuity"])
def test_zero_velocity_is_identity(model):
    n = (10, 12, 8)
    rng = np.random.default_rng(0)
    m0 = rng.standard_normal(n)
    v = np.zeros((3,) + n)
    mu = np.zeros(n)
    ms = forward_states(model, m0, v, 4, mu=mu)
    for m in ms:
        assert np.array_equal(m, m0)
    lams = adjoint_states(model, m0, v, 4, mu=mu)
    for l in lams:
        assert np.array_equal(l, m0)


def test_constant_velocity_departure_points_are_exact():
    n = (8, 8)
    h = 2 * np.pi / 8
    v = np.stack([np.full(n, 0.37), np.full(n, -1.1)])
    nt = 4
    xm = departure_points(v, nt, +1)
    xp = departure_points(v, nt, -1)
    base = grid_index(n)
    for a in range(2):
        np.testing.assert_allclose(xm[a], base[a] - v[a] / nt / h, atol=1e-14)
        np.testing.assert_allclose(xp[a], base[a] + v[a] / nt / h, atol=1e-14)


@pytest.mark.parametrize("model", ["advection", "continuity"])
def test_integer_shift_is_exact_roll(model):
    n = (16, 12, 10)
    nt = 4
    h = [2 * np.pi / k for k in n]
    cells = (1, -2, 3)  # cells moved per time step
    v = np.stack([np.full(n, cells[a] * h[a] * nt) for a in range(3)])
    rng = np.random.default_rng(1)
    m0 = rng.standard_normal(n)
    ms = forward_states(model, m0, v, nt, mu=np.zeros(n))
    for j, m in enumerate(ms):
        assert np.array_equal(m, np.roll(m0, tuple(c * j for c in cells), axis=(0, 1, 2)))
    lams = adjoint_states(model, m0, v, nt, mu=np.zeros(n))
    for j, l in enumerate(lams):
        assert np.array_equal(l, np.roll(m0, tuple(-c * (nt - j) for c in cells), axis=(0, 1, 2)))


def test_constant_velocity_matches_exact_shift_fourth_order():
    c = np.array([0.41, -0.23])
    errs = []
    for N in (16, 32, 64):
        n = (N, N)
        X = _grid(n)
        m0 = np.sin(X[0]) * np.cos(2 * X[1]) + 0.3 * np.cos(X[0] - X[1])
        exact = np.sin(X[0] - c[0]) * np.cos(2 * (X[1] - c[1])) + 0.3 * np.cos(X[0] - c[0] - X[1] + c[1])
        v = np.stack([np.full(n, c[0]), np.full(n, c[1])])
        mT = forward_states("advection", m0, v, 4, mu=np.zeros(n))[-1]
        errs.append(np.abs(mT - exact).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    # interpolation error O(h^4) only (RK2 characteristics are exact for constant v)
    assert rates[0] > 3.0 and rates[-1] > 3.6, (errs, rates)


def test_continuity_mass_drift_vanishes_under_refinement():
    # Mass (sum pi h^d) is preserved by the continuity equation (Sec. 3.7); the SL scheme
    # is not exactly conservative, so the pin is the rate at which the drift vanishes.
    drifts = []
    for N, nt in ((16, 2), (32, 4), (64, 8)):
        n = (N, N)
        X = _grid(n)
        pi0 = 1.0 + 0.5 * np.sin(X[0]) * np.cos(X[1])
        v = np.stack([0.4 * np.sin(X[1]) + 0.3 * np.cos(X[0]), 0.35 * np.cos(X[0] + X[1])])
        mu = sp.div(v)
        ms = forward_states("continuity", pi0, v, nt, mu=mu)
        drifts.append(abs(ms[-1].sum() - pi0.sum()) / pi0.sum())
    rates = np.log2(np.array(drifts[:-1]) / np.array(drifts[1:]))
    # h_t = 1/n_t is refined with h: the drift falls at second order (rate -> 2)
    assert np.all(rates > 1.5) and rates[-1] > 1.8, (drifts, rates)


def test_advection_of_divergence_free_field_keeps_mean_to_discretisation_error():
    # Under a divergence-free velocity the advection equation preserves the integral of m;
    # the discrete drift must vanish under refinement.
    drifts = []
    for N, nt in ((16, 4), (32, 8), (64, 16)):
        n = (N, N)
        X = _grid(n)
        m0 = np.sin(X[0]) ** 2 + np.cos(X[1])
        v = 0.5 * np.stack([np.sin(X[0]) * np.cos(X[1]), -np.cos(X[0]) * np.sin(X[1])])
        assert np.abs(sp.div(v)).max() < 1e-12
        mT = forward_states("advection", m0, v, nt)[-1]
        drifts.append(abs(mT.mean() - m0.mean()))
    rates = np.log2(np.array(drifts[:-1]) / np.array(drifts[1:]))
    assert np.all(rates > 1.5), (drifts, rates)


def test_adjoint_advection_source_matches_closed_form_for_linear_growth():
    # With v = 0 except a spatially constant divergence the adjoint ODE is d lambda/d tau =
    # lambda mu; check one Heun step on a constant field against the RK2 closed form.
    n = (8, 8)
    v = np.zeros((2,) + n)
    mu = np.full(n, 0.7)
    nt = 4
    ht = 1.0 / nt
    lam = adjoint_states("advection", np.ones(n), v, nt, mu=mu)
    factor = 1 + 0.5 * ht * (0.7 + 0.7 * (1 + ht * 0.7))
    for j in range(nt + 1):
        np.testing.assert_allclose(lam[j], factor ** (nt - j), rtol=1e-14)
    pis = forward_states("continuity", np.ones(n), v, nt, mu=mu)
    fwd = 1 - 0.5 * ht * (0.7 + 0.7 * (1 - ht * 0.7))
    for j in range(nt + 1):
        np.testing.assert_allclose(pis[j], fwd ** j, rtol=1e-14)


def test_point_restricted_steps_equal_the_full_grid():
    """The per-point departure points and state/adjoint steps (used for sampled parity at full size)
    give the full-grid values at any set of grid points."""
    from oracle.transport import adjoint_step_at, departure_points_at, state_step_at

    n = (10, 12, 8)
    rng = np.random.default_rng(9)
    v = random_fourier_field(n, 3, 3, rng) * 0.3
    m = rng.standard_normal(n)
    mu = sp.div(v)
    pts = np.stack([rng.integers(0, k, size=40) for k in n])
    xm_all = departure_points(v, 4, +1)
    xm = departure_points_at(v, 4, +1, pts)
    np.testing.assert_allclose(xm, xm_all[(slice(None),) + tuple(pts)], atol=1e-14)
    for model in ("advection", "continuity"):
        full = forward_states(model, m, v, 4, mu=mu)[1]
        np.testing.assert_allclose(state_step_at(model, m, mu, xm, pts, 4), full[tuple(pts)], atol=1e-13)
        xp = departure_points_at(v, 4, -1, pts)
        fulla = adjoint_states(model, m, v, 4, mu=mu)[3]
        np.testing.assert_allclose(adjoint_step_at(model, m, mu, xp, pts, 4), fulla[tuple(pts)], atol=1e-13)


# A flow with non-constant velocity whose characteristics are known in closed form (Sec. 2.2, the RK2
# characteristics): v = (a, b sin x_0) on a 2D periodic grid. Backward along v for a time h_t the
# departure point is x_0 - a h_t, x_1 - (b/a)(cos(x_0 - a h_t) - cos x_0); forward (the adjoint's
# characteristics of -v) it is x_0 + a h_t, x_1 + (b/a)(cos x_0 - cos(x_0 + a h_t)). With a = pi/2 on
# 256 cells, a h_t is a whole number of cells for n_t | 64, so I[v](X*) carries no interpolation error
# (v_1 depends on x_0 only) and the measured error is the time discretisation alone: one Heun step is
# the trapezoidal rule for the x_1 integral, local error O(h_t^3); forward Euler, or a predictor
# X* taken with the wrong sign, is O(h_t^2).
_RK2_N, _RK2_A, _RK2_B = (256, 8), np.pi / 2, 0.7


def _rk2_flow():
    X = _grid(_RK2_N)
    return X, np.stack([np.full(_RK2_N, _RK2_A), _RK2_B * np.sin(X[0])])


def _rk2_step_errors(sign):
    from oracle.transport import departure_points

    X, v = _rk2_flow()
    h = [2 * np.pi / k for k in _RK2_N]
    errs = []
    for nt in (4, 8, 16, 32):
        ht = 1.0 / nt
        xi = departure_points(v, nt, sign)
        a, b = _RK2_A, _RK2_B
        ex0 = X[0] - sign * a * ht
        ex1 = X[1] - (b / a) * (np.cos(X[0] - sign * a * ht) - np.cos(X[0]))
        errs.append(max(np.abs(xi[0] * h[0] - ex0).max(), np.abs(xi[1] * h[1] - ex1).max()))
    return np.array(errs)


@pytest.mark.parametrize("sign", [+1, -1])
def test_rk2_departure_points_third_order_on_closed_form_flow(sign):
    errs = _rk2_step_errors(sign)
    rates = np.log2(errs[:-1] / errs[1:])
    assert errs[0] < 5e-3, errs
    assert np.all(rates > 2.8) and np.all(rates < 3.2), (errs, rates)


@pytest.mark.parametrize("bad", ["euler", "predictor_sign"])
@pytest.mark.parametrize("sign", [+1, -1])
def test_rk2_pin_catches_planted_mistakes(monkeypatch, bad, sign):
    """The rate pin above fails for planted mistakes in the oracle's characteristics: a predictor
    value taken at x (forward Euler) or at the mirrored point x + sign h_t v (predictor sign slip)."""
    import oracle.transport as tr
    from oracle.interp import interp as true_interp

    pts = tr.grid_index(_RK2_N)

    def planted(f, xi):
        if bad == "euler":
            return true_interp(f, pts)
        return true_interp(f, 2 * pts - xi)

    monkeypatch.setattr(tr, "interp", planted)
    errs = _rk2_step_errors(sign)
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates < 2.3), (errs, rates)
