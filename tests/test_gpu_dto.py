"""GPU parity of the discretise-then-optimise gradient (the exact derivative of the discrete objective)
and of the exact transport vector-Jacobian product against the oracle (oracle/dto.py)."""
import numpy as np
import pytest

from gpu_util import TOL, TOL_GRAD_MIXED, empty, host, quantise, rel_l2, to_dev
from oracle import dto
from oracle import spectral as osp
from synth.inputs import random_fourier_field, random_problem_fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_08782_gb300 import build

    build.build()


def _setup(shape, prec, model, nt=3, s=1, alpha=1e-3, seed=0):
    from paper_2510_08782_gb300 import Problem

    m0, m1, v = random_problem_fields(shape, seed, model=model, vel_scale_vox=1.3)
    m0, m1, v = quantise(m0, prec), quantise(m1, prec), quantise(v, prec)
    P = Problem(to_dev(m0, prec), to_dev(m1, prec), nt=nt, model=model, reg_order=s, alpha=alpha, prec=prec)
    return P, m0, m1, v


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("model", ["advection", "incompressible"])
@pytest.mark.parametrize("shape", [(32, 24), (16, 12, 20), (20, 24, 18)])
def test_discrete_gradient_matches_oracle(shape, prec, model):
    P, m0, m1, v = _setup(shape, prec, model)
    g = empty(v.shape, prec)
    J = P.gradient_dto(to_dev(v, prec), g)
    gref = dto.gradient(m0, m1, v, 3, 1, 1e-3, model=model)
    Jref = dto.objective(m0, m1, v, 3, 1, 1e-3)
    tol = TOL[prec] if prec == "fp64" else TOL_GRAD_MIXED
    assert abs(J - Jref) <= tol * abs(Jref)
    assert rel_l2(host(g), gref) < tol, rel_l2(host(g), gref)


@pytest.mark.parametrize("shape", [(32, 24), (16, 12, 20)])
def test_discrete_gradient_is_the_derivative_of_the_gpu_objective(shape):
    """FP64: central differences of the library's own objective agree with it to their truncation
    error (the optimise-then-discretise gradient agrees only to discretisation error)."""
    P, m0, m1, v = _setup(shape, "fp64", "advection")
    g = empty(v.shape, "fp64")
    P.gradient_dto(to_dev(v, "fp64"), g)
    host_grad = host(g)
    rng = np.random.default_rng(8)
    fds, ans = [], []
    for _ in range(3):
        d = random_fourier_field(shape, len(shape), 3, rng)
        d /= np.abs(d).max()
        eps = 1e-7  # small enough that no departure point crosses a cell face (a kink of the interpolant)
        fds.append((P.objective(to_dev(v + eps * d, "fp64")) - P.objective(to_dev(v - eps * d, "fp64"))) / (2 * eps))
        ans.append(osp.inner(host_grad, d, shape))
    fds, ans = np.array(fds), np.array(ans)
    # relative to the largest directional derivative: the differences carry an absolute rounding floor
    assert np.abs(fds - ans).max() <= 1e-6 * np.abs(fds).max(), (fds, ans)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_exact_transport_vjp_and_autograd_backward(prec):
    from paper_2510_08782_gb300.autograd import transport

    shape = (16, 12, 10)
    P, m0, _, v = _setup(shape, prec, "advection")
    gamma = quantise(np.random.default_rng(3).standard_normal(shape), prec)
    ref = dto.transport_vjp(m0, v, 3, gamma)
    out = empty(v.shape, prec)
    P.transport_vjp(to_dev(v, prec), to_dev(gamma, prec), out, exact=True)
    tol = TOL[prec] if prec == "fp64" else 3 * TOL["mixed"]
    assert rel_l2(host(out), ref) < tol, rel_l2(host(out), ref)
    vt = to_dev(v, prec).requires_grad_(True)
    (transport(vt, P, exact=True) * to_dev(gamma, prec)).sum().backward()
    assert rel_l2(host(vt.grad), ref) < tol


def test_continuity_model_is_rejected():
    from paper_2510_08782_gb300 import GaError

    P, _, _, v = _setup((16, 12, 20), "fp64", "continuity")
    g = empty(v.shape, "fp64")
    with pytest.raises(GaError) as e:
        P.gradient_dto(to_dev(v, "fp64"), g)
    assert e.value.status == 1 and "advection" in str(e.value)
