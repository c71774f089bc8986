"""Pins of the oracle's discretise-then-optimise gradient: it is the exact derivative of the discrete
objective, so central differences agree with it to their truncation error, and it approaches the
paper's optimise-then-discretise gradient as the discretisation is refined (Sec. 2.1)."""
import numpy as np
import pytest

from oracle import dto
from oracle import spectral as sp
from oracle.interp import interp
from oracle.problem import Problem
from synth.inputs import random_fourier_field, random_problem_fields


def test_interpolant_derivative_matches_differences_inside_cells():
    rng = np.random.default_rng(1)
    f = rng.standard_normal((9, 11, 7))
    pts = np.stack([rng.uniform(0, k, size=200) for k in f.shape])
    pts = np.floor(pts) + np.clip(pts - np.floor(pts), 0.01, 0.99)  # keep the differences inside one cell
    g = dto.interp_grad(f, pts)
    eps = 1e-6
    for a in range(3):
        e = np.zeros((3, 1))
        e[a] = eps
        fd = (interp(f, pts + e) - interp(f, pts - e)) / (2 * eps)
        np.testing.assert_allclose(g[a], fd, rtol=0, atol=1e-7 * np.abs(f).max())


def test_interpolant_derivative_converges_at_third_order():
    """For sin(k x) the derivative of the cubic interpolant errs by O(h^3)."""
    errs = []
    for n in (16, 32, 64):
        x = 2 * np.pi * np.arange(n) / n
        f = np.sin(3 * x)
        pts = np.linspace(0.0, n, 97, endpoint=False)[None] + 0.37
        g = dto.interp_grad(f, pts)[0] * n / (2 * np.pi)  # per unit x
        errs.append(np.abs(g - 3 * np.cos(3 * 2 * np.pi * pts[0] / n)).max())
    assert errs[1] < errs[0] / 6 and errs[2] < errs[1] / 6, errs


@pytest.mark.parametrize("shape,nt,s", [((20, 16), 4, 1), ((12, 10, 8), 3, 2)])
def test_gradient_is_the_derivative_of_the_discrete_objective(shape, nt, s):
    m0, m1, v = random_problem_fields(shape, 5, vel_scale_vox=1.3)
    alpha = 1e-3
    g = dto.gradient(m0, m1, v, nt, s, alpha)
    rng = np.random.default_rng(2)
    for _ in range(4):
        d = random_fourier_field(shape, len(shape), 3, rng)
        d /= np.abs(d).max()
        eps = 1e-5
        fd = (dto.objective(m0, m1, v + eps * d, nt, s, alpha) - dto.objective(m0, m1, v - eps * d, nt, s, alpha)) / (
            2 * eps)
        an = sp.inner(g, d, shape)
        assert abs(fd - an) <= 1e-6 * abs(fd), (fd, an)


def test_transport_vjp_is_exact():
    shape, nt = (14, 12, 10), 3
    m0, _, v = random_problem_fields(shape, 6, vel_scale_vox=1.0)
    gamma = np.random.default_rng(3).standard_normal(shape)
    vjp = dto.transport_vjp(m0, v, nt, gamma)

    def mT(vv):
        from oracle.transport import forward_states

        return forward_states("advection", m0, vv, nt)[-1]

    d = random_fourier_field(shape, 3, 3, np.random.default_rng(4))
    d /= np.abs(d).max()
    eps = 1e-6  # small enough that no departure point crosses a cell face, where the interpolant has a kink
    fd = float(np.sum(gamma * (mT(v + eps * d) - mT(v - eps * d)))) / (2 * eps)
    assert abs(fd - float(np.sum(vjp * d))) <= 1e-6 * abs(fd)


def test_discrete_and_continuous_adjoint_gradients_converge_together():
    """The gap between this gradient and the paper's optimise-then-discretise one is a discretisation
    error: it shrinks when the grid and the time step are refined together."""
    gaps = []
    for n, nt in ((32, 4), (64, 8)):
        x = np.meshgrid(*[2 * np.pi * np.arange(n) / n] * 2, indexing="ij")
        m0 = np.sin(x[0]) * np.cos(2 * x[1]) + 0.5 * np.cos(x[0] + x[1])
        m1 = np.sin(x[0] - 0.3) * np.cos(2 * x[1] + 0.2) + 0.5 * np.cos(x[0] + x[1] - 0.1)
        v = np.stack([0.2 + 0.1 * np.sin(x[1]), -0.15 + 0.1 * np.cos(x[0])])
        g_dto = dto.gradient(m0, m1, v, nt, 1, 1e-3)
        g_otd, _ = Problem(m0, m1, nt=nt, model="advection", reg_order=1, alpha=1e-3).gradient(v)
        gaps.append(np.linalg.norm(g_dto - g_otd) / np.linalg.norm(g_otd))
    assert gaps[0] < 0.2 and gaps[1] < gaps[0] / 1.8, gaps
