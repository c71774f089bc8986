"""GPU parity of the solver (Alg. 3 with the Armijo map q of Eqs. (6)-(10)) against the oracle,
and the error paths of the C ABI that need a device (NaN input, exhausted line search)."""
import numpy as np
import pytest

from gpu_util import empty, host, quantise, rel_l2, to_dev
from oracle import solver as osol
from oracle.problem import Problem as OProblem
from synth.inputs import random_problem_fields, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_08782_gb300 import build

    build.build()


def _pair(w, prec, stream=None, **kw):
    from paper_2510_08782_gb300 import Problem

    m0, m1 = quantise(w["m0"], prec), quantise(w["m1"], prec)
    opts = dict(nt=w["nt"], model=w["model"], reg_order=w["reg_order"], alpha=w["alpha"])
    sopts = dict(window=w["window"], sigma=w["sigma"], tau=w["tau"], max_iter=w["max_iter"],
                 rel_tol=w["rel_tol"])
    sopts.update(kw)
    d0, d1 = to_dev(m0, prec), to_dev(m1, prec)
    if stream is not None:  # the context's stream does not order itself after the default stream
        import torch

        torch.cuda.synchronize()
    P = Problem(d0, d1, prec=prec, stream=stream, **opts, **sopts)
    O = OProblem(m0, m1, **opts)
    return P, O, sopts


@pytest.mark.parametrize("variant", [1, 2])
def test_iterates_match_oracle_fp64(variant):
    """First iterates of GA-NGMRES(5; 2, 1) (both mixing variants) on a small 2D advection problem:
    line-search decisions, window least squares and combination reproduce the oracle's iterates."""
    w = workload("adv2d64", n=(32, 32))
    P, O, so = _pair(w, "fp64", window=3, sigma=2, tau=1, max_iter=8, variant=variant)
    v = to_dev(np.zeros((2, 32, 32)), "fp64")
    hist = []
    q = osol.ArmijoQ(O)
    osol.ga_ngmres(O.gradient, q, np.zeros((2, 32, 32)), window=3, sigma=2, tau=1, n_iter=6,
                   rel_tol=0.0, variant=variant, history=hist)
    for k, h in enumerate(hist):
        st = P.step(v)
        assert st.iters == k + 1
        assert st.last_branch == (1 if h["branch"] == "fp" else 0)
        err = rel_l2(host(v), h["v"])
        assert err < 1e-8, (k, err)
        assert abs(st.obj - h["obj"]) <= 1e-9 * abs(h["obj"])
    assert abs(st.rho_mem - q.rho_mem) == 0.0


@pytest.mark.parametrize("variant,sigma,tau", [(1, 2, 1), (2, 2, 1), (1, 1, 1)])
def test_ga_aa_iterates_match_oracle_fp64(variant, sigma, tau):
    """GA-AA(3; sigma, tau) (Anderson acceleration on q with the mixing of Alg. 3): the residual
    window, its least squares and the combination of the q's reproduce the oracle's iterates."""
    w = workload("adv2d64", n=(32, 32))
    P, O, so = _pair(w, "fp64", window=3, sigma=sigma, tau=tau, max_iter=8, variant=variant, method="ga-aa")
    v = to_dev(np.zeros((2, 32, 32)), "fp64")
    hist = []
    q = osol.ArmijoQ(O)
    osol.ga_aa(O.gradient, q, np.zeros((2, 32, 32)), window=3, sigma=sigma, tau=tau, n_iter=7, rel_tol=0.0,
               variant=variant, history=hist)
    assert any(h["branch"] == "aa" for h in hist)
    for k, h in enumerate(hist):
        st = P.step(v)
        assert st.iters == k + 1
        assert st.last_branch == (1 if h["branch"] == "fp" else 0)
        err = rel_l2(host(v), h["v"])
        assert err < 1e-8, (k, err)
        assert abs(st.obj - h["obj"]) <= 1e-9 * abs(h["obj"])
    assert abs(st.rho_mem - q.rho_mem) == 0.0


def test_mixed_solver_carries_the_regulariser_on_a_512_axis():
    """H2 on a 512-point axis in mixed precision: the solver carries alpha L v through its linear
    updates instead of transforming its FP32 iterate, so its iterates and reported gradient norms
    follow the FP64 oracle's GA-NGMRES run step by step (a transform of v would put an O(1e-2)
    error into the gradient here, see test_gradient_with_a_512_axis)."""
    shape = (8, 12, 512)
    m0, m1, _ = random_problem_fields(shape, 21, vel_scale_vox=1.5)
    w = dict(m0=m0, m1=m1, nt=4, model="advection", reg_order=2, alpha=1e-3, window=5, sigma=4, tau=2,
             max_iter=10, rel_tol=0.0)
    P, O, so = _pair(w, "mixed")
    hist = []
    osol.ga_ngmres(O.gradient, osol.ArmijoQ(O), np.zeros((3,) + shape), window=5, sigma=4, tau=2, n_iter=6,
                   rel_tol=0.0, history=hist)
    v = to_dev(np.zeros((3,) + shape), "mixed")
    for k, h in enumerate(hist):
        st = P.step(v)
        assert rel_l2(host(v), h["v"]) < 2e-4, (k, rel_l2(host(v), h["v"]))
        assert abs(st.rel_grad_inf - h["rel_grad"]) <= 2e-3 * h["rel_grad"], (k, st.rel_grad_inf, h["rel_grad"])
        assert abs(st.obj - h["obj"]) <= 1e-4 * abs(h["obj"])


def test_ga_aa_window_zero_is_rpgd():
    """With w = 0 every GA-AA step is a fixed-point step, so the iterates are those of RPGD."""
    w = workload("adv2d64", n=(32, 32))
    P1, _, _ = _pair(w, "fp64", window=0, max_iter=5, method="ga-aa")
    P2, _, _ = _pair(w, "fp64", window=0, max_iter=5, method="rpgd")
    v1 = to_dev(np.zeros((2, 32, 32)), "fp64")
    v2 = to_dev(np.zeros((2, 32, 32)), "fp64")
    for _ in range(4):
        s1, s2 = P1.step(v1), P2.step(v2)
        assert s1.last_branch == 1 and s2.last_branch == 1
        assert np.array_equal(host(v1), host(v2))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_solve_matches_oracle_adv2d64(prec):
    """2D 64x64 advection workload (8 blobs, H1, alpha 1e-2, w 5, (4,2)), solved to rel-grad 1e-2."""
    w = workload("adv2d64")
    P, O, so = _pair(w, prec, max_iter=40)
    _, info = osol.solve_problem(O, window=5, sigma=4, tau=2, n_iter=40, rel_tol=1e-2)
    v = to_dev(np.zeros((2, 64, 64)), prec)
    st, status = P.solve(v)
    assert status == 0 and st.converged
    assert abs(st.iters - info["iters"]) <= (0 if prec == "fp64" else 2)
    assert st.rel_grad_inf <= 1e-2
    tol = 1e-6 if prec == "fp64" else 1e-3
    assert abs(st.obj - info["obj"]) <= tol * abs(info["obj"])


def test_rpgd_is_slower_than_ga_ngmres_on_gpu():
    w = workload("adv2d64")
    P1, _, _ = _pair(w, "fp64", max_iter=60)
    P2, _, _ = _pair(w, "fp64", max_iter=60, method="rpgd")
    v1 = to_dev(np.zeros((2, 64, 64)), "fp64")
    v2 = to_dev(np.zeros((2, 64, 64)), "fp64")
    s1, _ = P1.solve(v1)
    s2, _ = P2.solve(v2)
    assert s1.converged and s1.iters < s2.iters


def test_nan_input_is_reported():
    from paper_2510_08782_gb300 import GaError

    w = workload("adv2d64", n=(16, 16))
    P, _, _ = _pair(w, "fp64")
    v = np.zeros((2, 16, 16))
    v[0, 3, 4] = np.nan
    g = empty(v.shape, "fp64")
    with pytest.raises(GaError) as e:
        P.gradient(to_dev(v, "fp64"), g)
    assert e.value.status == 4
    # the context stays usable
    J = P.gradient(to_dev(np.zeros_like(v), "fp64"), g)
    assert np.isfinite(J)


def test_exhausted_line_search_is_reported():
    from paper_2510_08782_gb300 import GaError

    w = workload("adv2d64", n=(16, 16))
    P, _, _ = _pair(w, "fp64", armijo_c=1e30, max_backtracks=3)
    v = to_dev(np.zeros((2, 16, 16)), "fp64")
    with pytest.raises(GaError) as e:
        P.step(v)
    assert e.value.status == 5
    assert "Armijo" in str(e.value)


@pytest.mark.parametrize("model,method,shape,prec", [("advection", "ga-ngmres", (20, 16, 24), "mixed"),
                                                      ("continuity", "ga-ngmres", (16, 12, 20), "mixed"),
                                                      ("incompressible", "ga-ngmres", (16, 16, 16), "mixed"),
                                                      ("advection", "ga-aa", (32, 24), "fp64")])
def test_graph_replay_equals_kernel_by_kernel(model, method, shape, prec):
    """Capturing the solver's evaluations into CUDA graphs changes nothing: iterates and statistics of
    9 iterations are bitwise equal to kernel-by-kernel launches (every variant is first run eagerly,
    then captured, then replayed)."""
    m0, m1, _ = random_problem_fields(shape, 33, model=model, vel_scale_vox=1.2)
    w = dict(m0=m0, m1=m1, nt=4, model=model, reg_order=1, alpha=1e-2, window=4, sigma=2, tau=1, max_iter=20,
             rel_tol=0.0)
    P0, _, _ = _pair(w, prec, method=method)
    P1, _, _ = _pair(w, prec, method=method, graphs=True)
    v0 = to_dev(np.zeros((len(shape),) + shape), prec)
    v1 = to_dev(np.zeros((len(shape),) + shape), prec)
    for _ in range(9):
        s0, s1 = P0.step(v0), P1.step(v1)
        assert np.array_equal(host(v0), host(v1))
        assert (s0.obj, s0.rel_grad_inf, s0.last_branch, s0.ls_trials) == (s1.obj, s1.rel_grad_inf, s1.last_branch,
                                                                           s1.ls_trials)


@pytest.mark.parametrize("graphs", [False, True])
def test_batch_of_uneven_problems_matches_individual_solves(graphs):
    """The batched form: uneven problems, each on its own stream (and, with graphs, replaying its
    captured evaluations), solved concurrently, give the same iterates as one-at-a-time solves."""
    import torch

    from paper_2510_08782_gb300 import ga_solve_batch

    probs, vs, refs = [], [], []
    for i, n in enumerate([(16, 16, 16), (24, 24, 24), (20, 20, 20), (32, 24, 20)]):
        m0, m1, _ = random_problem_fields(n, 40 + i, vel_scale_vox=1.0)
        w = dict(m0=m0, m1=m1, nt=4, model="advection", reg_order=1, alpha=1e-2, window=5, sigma=4,
                 tau=2, max_iter=15, rel_tol=1e-2)
        P, _, _ = _pair(w, "mixed", stream=torch.cuda.Stream().cuda_stream, graphs=graphs)
        Q, _, _ = _pair(w, "mixed")
        probs.append(P)
        vs.append(to_dev(np.zeros((3,) + n), "mixed"))
        vq = to_dev(np.zeros((3,) + n), "mixed")
        refs.append((Q.solve(vq)[0], vq))
    torch.cuda.synchronize()
    stats, status = ga_solve_batch([p.ctx for p in probs], np.float32, vs)
    torch.cuda.synchronize()
    for st, (ref, vq), v in zip(stats, refs, vs):
        assert st.iters == ref.iters
        assert np.array_equal(host(v), host(vq))
