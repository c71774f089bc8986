"""Parity at the full sizes of the smaller named workloads (the 2D 64^2 and 3D 64^3 advection problems
and the 3D 128^3 incompressible problem), against the FP64 oracle through the C ABI and the autograd
wrapper."""
import numpy as np
import pytest

from gpu_util import TOL, TOL_GRAD_MIXED, empty, host, quantise, rel_l2, to_dev
from oracle import solver as osol
from oracle import spectral as osp
from oracle.problem import Problem as OProblem
from synth.inputs import random_fourier_field, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_08782_gb300 import build

    build.build()


def _problems(w, prec, **kw):
    from paper_2510_08782_gb300 import Problem

    m0, m1 = quantise(w["m0"], prec), quantise(w["m1"], prec)
    opts = dict(nt=w["nt"], model=w["model"], reg_order=w["reg_order"], alpha=w["alpha"])
    sopts = dict(window=w["window"], sigma=w["sigma"], tau=w["tau"], max_iter=w["max_iter"], rel_tol=w["rel_tol"])
    sopts.update(kw)
    return Problem(to_dev(m0, prec), to_dev(m1, prec), prec=prec, **opts, **sopts), OProblem(m0, m1, **opts)


def test_adv2d64_twenty_iterations_match_oracle():
    """2D 64^2 advection, FP64, GA-NGMRES(5; 4, 2), 20 iterations: every iterate, branch and objective
    value against the oracle's Alg. 3 run."""
    w = workload("adv2d64")
    P, O = _problems(w, "fp64")
    hist = []
    osol.ga_ngmres(O.gradient, osol.ArmijoQ(O), np.zeros((2, 64, 64)), window=5, sigma=4, tau=2, n_iter=20,
                   rel_tol=0.0, history=hist)
    assert len(hist) == 20
    v = to_dev(np.zeros((2, 64, 64)), "fp64")
    for k, h in enumerate(hist):
        st = P.step(v)
        assert st.last_branch == (1 if h["branch"] == "fp" else 0), k
        assert rel_l2(host(v), h["v"]) < 1e-8, (k, rel_l2(host(v), h["v"]))
        assert abs(st.obj - h["obj"]) <= 1e-9 * abs(h["obj"]), k


def test_adv3d64_gradient_matches_oracle_at_full_size():
    """3D 64^3 advection, H2, alpha 1e-3, FP64: the reduced gradient and objective at half the true
    velocity, element by element."""
    w = workload("adv3d64")
    P, O = _problems(w, "fp64")
    v = 0.5 * w["v_true"]
    g = empty(v.shape, "fp64")
    J = P.gradient(to_dev(v, "fp64"), g)
    gref, Jref = O.gradient(v)
    assert abs(J - Jref) <= TOL["fp64"] * abs(Jref)
    assert rel_l2(host(g), gref) < TOL["fp64"], rel_l2(host(g), gref)


def test_adv3d64_ga_ngmres_needs_fewer_iterations_than_rpgd():
    """The comparison the 64^3 workload is defined by: GA-NGMRES and RPGD, both to rel-grad 1e-2 or
    200 iterations, FP64."""
    w = workload("adv3d64")
    P1, _ = _problems(w, "fp64")
    P2, _ = _problems(w, "fp64", method="rpgd")
    v1 = to_dev(np.zeros((3, 64, 64, 64)), "fp64")
    v2 = to_dev(np.zeros((3, 64, 64, 64)), "fp64")
    s1, _ = P1.solve(v1)
    s2, _ = P2.solve(v2)
    assert s1.converged and s1.rel_grad_inf <= 1e-2
    assert s1.iters < s2.iters, (s1.iters, s2.iters)


def test_inc128_autograd_gradient_and_fd_directions_at_full_size():
    """3D 128^3 incompressible workload, FP32 transport: the autograd backward of the data term equals
    the oracle's projected body force (after projecting the autograd gradient, which is the Euclidean
    gradient h^3 b), and its directional derivatives along 16 random divergence-free directions agree
    with central differences (eps 1e-4) of the FP64 objective to the discretisation error of the
    optimise-then-discretise gradient."""
    import torch

    from paper_2510_08782_gb300 import Problem
    from paper_2510_08782_gb300.autograd import transport

    w = workload("inc3d128")
    n = (128, 128, 128)
    m0, m1 = quantise(w["m0"], "mixed"), quantise(w["m1"], "mixed")
    v = quantise(osp.leray(0.5 * w["v_true"]), "mixed")
    P = Problem(to_dev(m0, "mixed"), to_dev(m1, "mixed"), nt=8, model="incompressible", reg_order=1, alpha=1e-2,
                prec="mixed")
    hd = osp.cell_volume(n)
    vt = to_dev(v, "mixed").requires_grad_(True)
    loss = 0.5 * hd * ((transport(vt, P) - to_dev(m1, "mixed")) ** 2).sum()
    loss.backward()
    ga = host(vt.grad)
    del vt, loss
    torch.cuda.empty_cache()
    O = OProblem(m0, m1, nt=8, model="incompressible", reg_order=1, alpha=1e-2)
    _, _, parts = O.gradient(v, return_parts=True)
    assert rel_l2(osp.leray(ga / hd), parts["body"]) < TOL_GRAD_MIXED, rel_l2(osp.leray(ga / hd), parts["body"])
    # central differences of the data term with the FP64 objective (regulariser switched off)
    P64 = Problem(to_dev(m0, "fp64"), to_dev(m1, "fp64"), nt=8, model="incompressible", reg_order=1, alpha=1e-30,
                  prec="fp64")
    rng = np.random.default_rng(11)
    fds, ans = [], []
    for _ in range(16):
        d = osp.leray(random_fourier_field(n, 3, 4, rng))
        d /= np.abs(d).max()
        eps = 1e-4
        fds.append((P64.objective(to_dev(v + eps * d, "fp64")) - P64.objective(to_dev(v - eps * d, "fp64"))) / (2 * eps))
        ans.append(float(np.sum(ga * d)))
    fds, ans = np.array(fds), np.array(ans)
    # the discretisation error of the gradient is absolute: measure it against the largest directional
    # derivative (a direction nearly orthogonal to the gradient has a tiny one), and bound the typical
    # relative error
    err = np.abs(fds - ans)
    assert err.max() < 0.05 * np.abs(fds).max(), (fds, ans)
    assert np.median(err / np.abs(fds)) < 0.02, (fds, ans)
