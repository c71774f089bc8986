"""GPU parity of the deformation diagnostics (the map y = x + h u and det grad y shown with the results
of Sec. 3) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from gpu_util import TOL, empty, host, quantise, rel_l2, to_dev
from oracle import spectral as osp
from oracle.diagnostics import deformation_displacement, det_grad_y
from synth.inputs import random_problem_fields, smooth_velocity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_08782_gb300 import build

    build.build()


def _problem(shape, prec, model="advection", nt=4):
    from paper_2510_08782_gb300 import Problem

    m0, m1, v = random_problem_fields(shape, 7, model=model, vel_scale_vox=1.5)
    m0, m1, v = quantise(m0, prec), quantise(m1, prec), quantise(v, prec)
    P = Problem(to_dev(m0, prec), to_dev(m1, prec), nt=nt, model=model, reg_order=1, alpha=1e-3, prec=prec)
    return P, v


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [(32, 24), (16, 12, 20), (36, 40, 48)])
def test_deformation_matches_oracle(shape, prec):
    """u and det grad y element by element on grids spanning several tiles with ragged edges."""
    nt = 6 if len(shape) == 2 else 4
    P, v = _problem(shape, prec, nt=nt)
    u = empty(v.shape, prec)
    dj = empty(shape, prec)
    P.deformation(to_dev(v, prec), u, dj)
    uref = deformation_displacement(v, nt)
    jref = det_grad_y(v, nt)
    tol = TOL[prec]
    assert rel_l2(host(u), uref) < tol, rel_l2(host(u), uref)
    assert rel_l2(host(dj), jref) < tol, rel_l2(host(dj), jref)
    # the deformation part of det grad y (det - 1) to the same relative accuracy in FP64, and
    # within FP32 rounding of the O(1) field in mixed precision
    err = np.abs(host(dj) - jref).max()
    assert err < (1e-11 if prec == "fp64" else 2e-5) * max(1.0, np.abs(jref - 1.0).max()), err


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_divergence_free_velocity_gives_unit_determinant(prec):
    """Incompressible flow (Sec. 3.6): det grad y = 1 up to rounding on the GPU as well."""
    from paper_2510_08782_gb300 import Problem

    shape = (24, 20, 30)
    rng = np.random.default_rng(5)
    v = quantise(osp.leray(smooth_velocity(shape, 4, 2.0, rng, divergence_free=True)), prec)
    m = quantise(np.ones(shape), prec)
    P = Problem(to_dev(m, prec), to_dev(m, prec), nt=4, model="incompressible", reg_order=3, alpha=1e-2, prec=prec)
    u = empty(v.shape, prec)
    dj = empty(shape, prec)
    P.deformation(to_dev(v, prec), u, dj)
    dev = np.abs(host(dj) - 1.0).max()
    assert dev < (1e-12 if prec == "fp64" else 1e-5), dev


def test_host_buffers_and_model_do_not_change_the_result():
    """Host and device buffers give bitwise equal outputs, and the diagnostics do not depend on the
    context's transport model."""
    shape = (16, 12, 20)
    P, v = _problem(shape, "mixed", model="advection")
    Q, _ = _problem(shape, "mixed", model="continuity")
    u_d, j_d = empty(v.shape, "mixed"), empty(shape, "mixed")
    P.deformation(to_dev(v, "mixed"), u_d, j_d)
    u_h = np.zeros(v.shape, dtype=np.float32)
    j_h = np.zeros(shape, dtype=np.float32)
    P.deformation(np.ascontiguousarray(v, dtype=np.float32), u_h, j_h)
    assert np.array_equal(host(u_d), u_h) and np.array_equal(host(j_d), j_h)
    u_q, j_q = empty(v.shape, "mixed"), empty(shape, "mixed")
    Q.deformation(to_dev(v, "mixed"), u_q, j_q)
    assert np.array_equal(host(u_q), u_h) and np.array_equal(host(j_q), j_h)
