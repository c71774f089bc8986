"""The device-driven solve (ga_solver_opts.graphs = 2): a whole solve, or a whole batch of solves, is one
CUDA graph launch whose conditional nodes take the line-search (Eqs. (6)-(7)) and step-kind (Alg. 3)
decisions on the device. It must reproduce the host-driven solver bit for bit: the same kernels run in
the same order on the same data, and the control kernels repeat the host's FP64 decisions."""
import numpy as np
import pytest

from gpu_util import host, to_dev
from synth.inputs import random_problem_fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_08782_gb300 import build

    build.build()


def _problem(shape, model, prec, seed=33, stream=None, **kw):
    from paper_2510_08782_gb300 import Problem

    m0, m1, _ = random_problem_fields(shape, seed, model=model, vel_scale_vox=1.2)
    dt = np.float64 if prec == "fp64" else np.float32
    opts = dict(nt=4, model=model, reg_order=1, alpha=1e-2, window=4, sigma=2, tau=1, max_iter=20, rel_tol=0.0)
    opts.update(kw)
    if stream is not None:  # the context's stream does not order itself after the default stream
        import torch

        torch.cuda.synchronize()
    return Problem(to_dev(m0.astype(dt), prec), to_dev(m1.astype(dt), prec), prec=prec, stream=stream, **opts)


FIELDS = ("iters", "grad_evals", "obj_evals", "pde_solves", "ls_trials", "last_branch", "converged", "obj",
          "mismatch", "rel_grad_inf", "grad_inf0", "rho_mem", "last_rho")


def _same_stats(a, b):
    for f in FIELDS:
        assert getattr(a, f) == getattr(b, f), (f, getattr(a, f), getattr(b, f))


CASES = [("advection", "ga-ngmres", (32, 24), "fp64", 1),
         ("advection", "ga-ngmres", (32, 24), "fp64", 2),
         ("advection", "rpgd", (24, 20), "fp64", 1),
         ("advection", "ga-ngmres", (20, 16, 24), "mixed", 1),
         ("continuity", "ga-ngmres", (16, 12, 20), "mixed", 1),
         ("incompressible", "ga-ngmres", (16, 16, 16), "mixed", 2)]


@pytest.mark.parametrize("model,method,shape,prec,variant", CASES)
def test_device_driven_solve_equals_host_driven(model, method, shape, prec, variant):
    P0 = _problem(shape, model, prec, method=method, variant=variant, max_iter=12)
    P2 = _problem(shape, model, prec, method=method, variant=variant, max_iter=12, graphs="device")
    v0 = to_dev(np.zeros((len(shape),) + shape), prec)
    v2 = to_dev(np.zeros((len(shape),) + shape), prec)
    s0, st0 = P0.solve(v0)
    s2, st2 = P2.solve(v2)
    assert st0 == st2
    assert np.array_equal(host(v0), host(v2))
    _same_stats(s0, s2)
    assert s2.iters == 12 and s2.ls_trials >= 12
    # a second solve from the same start replays the same graph and gives the same result
    v3 = to_dev(np.zeros((len(shape),) + shape), prec)
    s3, _ = P2.solve(v3)
    assert np.array_equal(host(v3), host(v2))
    _same_stats(s3, s2)


@pytest.mark.parametrize("model,shape,prec", [("advection", (32, 24), "fp64"), ("continuity", (16, 12, 20), "mixed")])
def test_device_driven_steps_equal_host_steps(model, shape, prec):
    """ga_step runs one iteration of the graph; seven of them track seven host-driven steps exactly,
    and a reset starts again from the caller's v."""
    P0 = _problem(shape, model, prec)
    P2 = _problem(shape, model, prec, graphs="device")
    for _ in range(2):
        v0 = to_dev(np.zeros((len(shape),) + shape), prec)
        v2 = to_dev(np.zeros((len(shape),) + shape), prec)
        for _ in range(7):
            s0, s2 = P0.step(v0), P2.step(v2)
            assert np.array_equal(host(v0), host(v2))
            _same_stats(s0, s2)
        P0.reset()
        P2.reset()


def test_device_driven_solve_stops_at_tolerance():
    P0 = _problem((32, 32), "advection", "fp64", rel_tol=1e-2, max_iter=50)
    P2 = _problem((32, 32), "advection", "fp64", rel_tol=1e-2, max_iter=50, graphs="device")
    v0 = to_dev(np.zeros((2, 32, 32)), "fp64")
    v2 = to_dev(np.zeros((2, 32, 32)), "fp64")
    s0, st0 = P0.solve(v0)
    s2, st2 = P2.solve(v2)
    assert s2.converged == 1 and st2 == st0 == 0 and s2.rel_grad_inf <= 1e-2
    assert s2.iters == s0.iters < 50
    assert np.array_equal(host(v0), host(v2))


def test_one_launch_batch_matches_individual_solves():
    """Uneven problems of both precisions, every one device-driven: the whole batch is one graph launch
    (kept and replayed by a second call) and each result equals the problem's own host-driven solve."""
    import torch

    from paper_2510_08782_gb300 import ga_solve_batch

    shapes = [(16, 16, 16), (24, 24, 24), (20, 20, 20), (32, 24, 20)]
    probs, refs = [], []
    for i, n in enumerate(shapes):
        kw = dict(seed=40 + i, window=5, sigma=4, tau=2, max_iter=15, rel_tol=1e-2)
        probs.append(_problem(n, "advection", "mixed", stream=torch.cuda.Stream().cuda_stream, graphs="device",
                              **kw))
        Q = _problem(n, "advection", "mixed", **kw)
        vq = to_dev(np.zeros((3,) + n), "mixed")
        refs.append((Q.solve(vq)[0], vq))
    torch.cuda.synchronize()
    for _ in range(2):
        vs = [to_dev(np.zeros((3,) + n), "mixed") for n in shapes]
        stats, status = ga_solve_batch([p.ctx for p in probs], np.float32, vs)
        torch.cuda.synchronize()
        assert status in (0, 6)
        for st, (ref, vq), v in zip(stats, refs, vs):
            _same_stats(st, ref)
            assert np.array_equal(host(v), host(vq))


def test_device_driven_failures_are_reported():
    from paper_2510_08782_gb300 import GaError

    P = _problem((16, 16), "advection", "fp64", armijo_c=1e30, max_backtracks=3, graphs="device")
    v = to_dev(np.zeros((2, 16, 16)), "fp64")
    with pytest.raises(GaError) as e:
        P.step(v)
    assert e.value.status == 5 and "Armijo" in str(e.value)
    assert P.stats().ls_trials == 4
    P2 = _problem((16, 16), "advection", "fp64", graphs="device")
    vn = np.zeros((2, 16, 16))
    vn[0, 3, 4] = np.nan
    with pytest.raises(GaError) as e:
        P2.solve(to_dev(vn, "fp64"))
    assert e.value.status == 4
    # the context stays usable: a clean start solves
    s, _ = P2.solve(to_dev(np.zeros((2, 16, 16)), "fp64"))
    assert s.iters == 20
