"""The batched form (ga_solve_batch, row a14) against the FP64 oracle, in both of its forms: one host
worker and stream per problem (graphs off), and the whole batch as one CUDA graph launch with the
solver's decisions on the device (graphs = 'device').

* FP64, uneven small grids: every member's first GA-NGMRES iterates (Alg. 3) equal the oracle's.
* Mixed precision at the batch workload's own sizes (64^3 and 96^3 members of the seeded batch of
  uneven advection problems, with a 128^3 member alongside): the first GA-NGMRES iterate of each
  checked member against the oracle. At k = 0 Alg. 3 takes an NGMRES step over the one-element window
  {v^(0) = 0}: q = q(v^(0)) = rho s(0), beta_0 = argmin ||g(q) + beta_0 (g(q) - g(0))||, and
  v^(1) = q + beta_0 (q - v^(0)). At v = 0 the oracle's gradient has a closed form (every state is m0 and
  every adjoint m1 - m0, the trapezoid weights sum to one), g(0) = (m1 - m0) grad m0, so s(0) =
  -(alpha L)^{-1} g(0) costs two transforms; the accepted step rho must pass the oracle's Armijo test
  (Eq. (7)) and, when it was halved, 2 rho must fail it.
"""
import numpy as np
import pytest

from gpu_util import TOL_GRAD_MIXED, host, quantise, rel_l2, to_dev
from oracle import solver as osol
from oracle import spectral as sp
from oracle.problem import Problem as OProblem
from synth.inputs import batch_problem, batch_specs, random_problem_fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_08782_gb300 import build

    build.build()


def _contexts(datas, prec, graphs, **kw):
    import torch

    from paper_2510_08782_gb300 import Problem

    probs = []
    for w in datas:
        st = torch.cuda.Stream()
        d0, d1 = to_dev(quantise(w["m0"], prec), prec), to_dev(quantise(w["m1"], prec), prec)
        torch.cuda.synchronize()  # the context's stream does not order itself after the default stream
        probs.append(Problem(d0, d1, nt=4, model="advection", reg_order=1, alpha=w["alpha"], prec=prec, window=5,
                             sigma=4, tau=2, stream=st.cuda_stream, graphs=graphs, **kw))
    return probs


@pytest.mark.parametrize("graphs", [False, "device"])
def test_batch_members_follow_the_oracle_fp64(graphs):
    from paper_2510_08782_gb300 import ga_solve_batch

    shapes = [(16, 16, 16), (24, 20, 16), (20, 20, 20), (32, 24, 20)]
    datas = []
    for i, n in enumerate(shapes):
        m0, m1, _ = random_problem_fields(n, 60 + i, vel_scale_vox=1.0)
        datas.append(dict(m0=m0, m1=m1, alpha=(1e-2, 1e-3)[i % 2]))
    iters = 4
    probs = _contexts(datas, "fp64", graphs, max_iter=iters, rel_tol=0.0)
    vs = [to_dev(np.zeros((3,) + n), "fp64") for n in shapes]
    stats, status = ga_solve_batch([p.ctx for p in probs], np.float64, vs)
    assert status in (0, 6)
    for w, n, st, v in zip(datas, shapes, stats, vs):
        O = OProblem(w["m0"], w["m1"], nt=4, model="advection", reg_order=1, alpha=w["alpha"])
        hist = []
        osol.ga_ngmres(O.gradient, osol.ArmijoQ(O), np.zeros((3,) + n), window=5, sigma=4, tau=2, n_iter=iters,
                       rel_tol=0.0, history=hist)
        assert st.iters == iters == len(hist)
        assert rel_l2(host(v), hist[-1]["v"]) < 1e-8, (n, rel_l2(host(v), hist[-1]["v"]))
        assert abs(st.obj - hist[-1]["obj"]) <= 1e-9 * abs(hist[-1]["obj"])
        assert st.last_branch == (1 if hist[-1]["branch"] == "fp" else 0)


@pytest.fixture(scope="module")
def batch_members():
    """The first 64^3, 96^3 and 128^3 members of the seeded batch of 32 (seed 0)."""
    picked = {}
    for spec in batch_specs(32, seed=0):
        if spec[1] in (64, 96, 128) and spec[1] not in picked:
            picked[spec[1]] = spec
    return [batch_problem(picked[k]) for k in (64, 96, 128)]


_ORACLE_FIRST = {}


def _oracle_first_iterate(w, rho):
    """The oracle's first GA-NGMRES iterate of member w for the accepted step rho (cached: both batched
    forms give the same rho), with the Armijo decisions checked."""
    key = (w["name"], rho)
    if key not in _ORACLE_FIRST:
        m0, m1 = quantise(w["m0"], "mixed"), quantise(w["m1"], "mixed")
        O = OProblem(m0, m1, nt=4, model="advection", reg_order=1, alpha=w["alpha"])
        g0 = (m1 - m0) * sp.grad(m0)  # closed form of the reduced gradient at v = 0
        s0 = O.precond(g0)
        obj0 = 0.5 * O.hd * float(np.sum((m0 - m1) ** 2))
        slope = O.inner(g0, s0)
        q = rho * s0
        gq, objq = O.gradient(q)
        assert objq < obj0 + 1e-4 * rho * slope  # the accepted step passes the oracle's Armijo test
        if rho < 1.0:  # the first trial of a solve is rho = 1; a halved step means 2 rho failed
            assert O.objective(2.0 * q) >= obj0 + 1e-4 * 2.0 * rho * slope - 1e-6 * abs(obj0)
        beta = osol.ngmres_lsq(gq, [g0])
        _ORACLE_FIRST[key] = (O, q + beta[0] * q)
    return _ORACLE_FIRST[key]


@pytest.mark.parametrize("graphs", [False, "device"])
def test_batch_first_iterate_at_batch_sizes_mixed(graphs, batch_members):
    from paper_2510_08782_gb300 import ga_solve_batch

    probs = _contexts(batch_members, "mixed", graphs, max_iter=1, rel_tol=0.0)
    vs = [to_dev(np.zeros((3,) + tuple(w["n"])), "mixed") for w in batch_members]
    stats, status = ga_solve_batch([p.ctx for p in probs], np.float32, vs)
    assert status in (0, 6)
    for w, st, v in zip(batch_members[:2], stats[:2], vs[:2]):  # the 64^3 and 96^3 members
        assert st.iters == 1 and st.last_rho > 0 and st.last_branch == 0
        O, v1_ref = _oracle_first_iterate(w, st.last_rho)
        v1 = host(v)
        assert rel_l2(v1, v1_ref) < TOL_GRAD_MIXED, (w["n"], rel_l2(v1, v1_ref))
        obj1 = O.objective(v1)
        assert abs(st.obj - obj1) <= 1e-4 * abs(obj1), (st.obj, obj1)
