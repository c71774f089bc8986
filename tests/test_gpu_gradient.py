"""GPU parity of the objective, reduced gradient and preconditioner (Eqs. (1a), (3), (9)) and of
the autograd transport wrapper, against the FP64 oracle, for the three models in 2D and 3D."""
import numpy as np
import pytest

from gpu_util import TOL, TOL_GRAD_MIXED, empty, host, quantise, rel_l2, to_dev
from oracle import spectral as osp
from oracle.problem import Problem as OProblem
from synth.inputs import random_fourier_field, random_problem_fields

pytestmark = pytest.mark.gpu

MODELS = ["advection", "continuity", "incompressible"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_08782_gb300 import build

    build.build()


def _setup(shape, prec, model, nt=4, s=2, alpha=1e-3, seed=0, ckpt=0):
    from paper_2510_08782_gb300 import Problem

    m0, m1, v = random_problem_fields(shape, seed, model=model, vel_scale_vox=1.5)
    m0, m1, v = quantise(m0, prec), quantise(m1, prec), quantise(v, prec)
    P = Problem(to_dev(m0, prec), to_dev(m1, prec), nt=nt, model=model, reg_order=s, alpha=alpha,
                prec=prec, ckpt_every=ckpt)
    O = OProblem(m0, m1, nt=nt, model=model, reg_order=s, alpha=alpha)
    return P, O, v


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("shape", [(32, 24), (16, 12, 20), (24, 20, 18)])
def test_objective_and_gradient(shape, prec, model):
    s = 1 if model != "advection" else 2
    P, O, v = _setup(shape, prec, model, s=s, nt=4 if len(shape) == 3 else 6)
    g = empty(v.shape, prec)
    J = P.gradient(to_dev(v, prec), g)
    gref, Jref = O.gradient(v)
    tol = TOL[prec] if prec == "fp64" else TOL_GRAD_MIXED
    assert abs(J - Jref) <= tol * abs(Jref)
    assert rel_l2(host(g), gref) < tol, rel_l2(host(g), gref)
    Jo = P.objective(to_dev(v, prec))
    assert abs(Jo - Jref) <= tol * abs(Jref)
    s_out = empty(v.shape, prec)
    P.precond(g, s_out)
    assert rel_l2(host(s_out), O.precond(host(g))) < TOL[prec] * 10


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [(16, 24, 256), (256, 16, 20), (16, 256, 20)])
def test_benchmark_path_gradient_at_nonzero_velocity(shape, prec):
    """The benchmark's configuration away from v = 0, on grids with a 256-point axis along each
    direction: continuity, n_t = 16, checkpoints every 4 steps, H1, alpha = 1e-3. The whole gradient runs
    the tiled transport steps (brick depth from the setup autotuner), the segment recompute of the
    backward sweep and the register-resident derivative passes; gradient and objective against the
    oracle."""
    P, O, v = _setup(shape, prec, "continuity", s=1, alpha=1e-3, nt=16, seed=5, ckpt=4)
    g = empty(v.shape, prec)
    J = P.gradient(to_dev(v, prec), g)
    gref, Jref = O.gradient(v)
    tol = TOL[prec] if prec == "fp64" else TOL_GRAD_MIXED
    assert abs(J - Jref) <= tol * abs(Jref)
    assert rel_l2(host(g), gref) < tol, rel_l2(host(g), gref)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [(32, 24), (16, 12, 20), (20, 24, 16)])
def test_incompressible_h3_gradient_and_preconditioner(shape, prec):
    """The incompressible runs of Sec. 3.6 use the H3 seminorm (L^ = |k|^6): gradient alpha L v + P b,
    objective, and the projected preconditioner s = -(alpha L)^{-1} P g against the oracle."""
    P, O, v = _setup(shape, prec, "incompressible", s=3, alpha=1e-4, nt=16 if len(shape) == 2 else 4, seed=3)
    g = empty(v.shape, prec)
    J = P.gradient(to_dev(v, prec), g)
    gref, Jref = O.gradient(v)
    tol = TOL[prec] if prec == "fp64" else TOL_GRAD_MIXED
    if prec == "mixed":  # alpha L v from an FP32 transform of the caller's v (see the 512-axis test below)
        L = osp.symbol_L(shape, 3)
        amp = 1e-4 * np.sqrt(np.mean(L ** 2)) * np.linalg.norm(v.ravel())
        tol += 6e-8 * np.log2(np.prod(shape)) * amp / np.linalg.norm(gref.ravel())
    assert abs(J - Jref) <= max(tol, TOL_GRAD_MIXED) * abs(Jref)
    assert rel_l2(host(g), gref) < tol, rel_l2(host(g), gref)
    s_out = empty(v.shape, prec)
    P.precond(g, s_out)
    sref = O.precond(host(g))
    assert rel_l2(host(s_out), sref) < TOL[prec] * 10
    assert np.abs(osp.div(sref)).max() < 1e-10 * np.abs(sref).max()  # the direction stays divergence free


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("model", ["advection", "continuity"])
def test_gradient_with_a_512_axis(prec, model):
    """A 512-point axis (the runtime-planned transform length of the 512^3 mesh study), H2. At a
    caller's v the mixed path must transform v to form alpha L v, and the FP32 rounding of that
    transform (about eps32 log2(N) |v| per coefficient) is multiplied by L^ = |k|^4, up to 256^4 here:
    the bound below states that, and the solver avoids it by carrying alpha L v (see test_gpu_solver)."""
    shape = (8, 12, 512)
    P, O, v = _setup(shape, prec, model, s=2, nt=4)
    g = empty(v.shape, prec)
    J = P.gradient(to_dev(v, prec), g)
    gref, Jref = O.gradient(v)
    tol = TOL[prec] if prec == "fp64" else TOL_GRAD_MIXED
    if prec == "mixed":
        L = osp.symbol_L(shape, 2)
        amp = 1e-3 * np.sqrt(np.mean(L ** 2)) * np.linalg.norm(v.ravel())  # alpha sqrt(mean L^2) |v|
        tol += 6e-8 * np.log2(np.prod(shape)) * amp / np.linalg.norm(gref.ravel())
    assert abs(J - Jref) <= max(tol, TOL_GRAD_MIXED) * abs(Jref)
    assert rel_l2(host(g), gref) < tol, (rel_l2(host(g), gref), tol)


@pytest.mark.parametrize("prec,nt,ckpt", [("fp64", 7, 1), ("fp64", 7, 3), ("fp64", 7, 4), ("mixed", 16, 4),
                                          ("mixed", 9, 4), ("mixed", 10, 3)])
def test_checkpointed_gradient_equals_stored(prec, nt, ckpt):
    """Checkpoints every K steps; the backward sweep recomputes each segment but the last, whose states
    the forward sweep left in the segment buffer. Recomputation repeats the same kernels on the same
    inputs, so the gradient is bitwise that of the stored trajectory (also through the solver's reuse
    of a line-search state solve)."""
    shape = (16, 12, 20)
    P0, O, v = _setup(shape, prec, "continuity", nt=nt, s=1)
    Pk, _, _ = _setup(shape, prec, "continuity", nt=nt, s=1, ckpt=ckpt)
    g0, gk = empty(v.shape, prec), empty(v.shape, prec)
    J0 = P0.gradient(to_dev(v, prec), g0)
    Jk = Pk.gradient(to_dev(v, prec), gk)
    assert J0 == Jk
    assert np.array_equal(host(g0), host(gk))
    v0 = to_dev(np.zeros_like(v), prec)
    vk = to_dev(np.zeros_like(v), prec)
    for _ in range(3):
        s0, sk = P0.step(v0), Pk.step(vk)
        assert np.array_equal(host(v0), host(vk)) and s0.obj == sk.obj


@pytest.mark.parametrize("model,nt,ckpt", [("continuity", 16, 4), ("advection", 9, 3), ("continuity", 7, 0)])
def test_overlapped_body_force_repeats_bitwise(model, nt, ckpt):
    """The body force's derivative passes run on a second stream of the context while the adjoint
    steps and segment recomputes go on in the first; adjoint states rotate through a ring of buffers and
    recomputed segments through two, each written again only after the passes that read it are done. A
    missing wait would let a pass read a buffer being overwritten in some calls and not in others: forty
    gradients on a grid where the kernels do overlap are bitwise equal to the first, and with
    checkpoints to the gradient of the stored trajectory."""
    from paper_2510_08782_gb300 import Problem

    shape, prec = (96, 96, 96), "mixed"
    m0, m1, v = random_problem_fields(shape, 5, model=model, vel_scale_vox=3.0)
    m0, m1, v = quantise(m0, prec), quantise(m1, prec), quantise(v, prec)

    def problem(k):
        return Problem(to_dev(m0, prec), to_dev(m1, prec), nt=nt, model=model, reg_order=1, alpha=1e-3,
                       prec=prec, ckpt_every=k)

    P = problem(ckpt)
    vd = to_dev(v, prec)
    g0 = empty(v.shape, prec)
    J0 = P.gradient(vd, g0)
    ref = host(g0)
    g = empty(v.shape, prec)
    for _ in range(40):
        assert P.gradient(vd, g) == J0
        assert np.array_equal(host(g), ref)
    if ckpt:
        Ps = problem(0)
        gs = empty(v.shape, prec)
        assert Ps.gradient(vd, gs) == J0
        assert np.array_equal(host(gs), ref)


def test_host_buffers_match_device_buffers():
    shape = (32, 24)
    P, O, v = _setup(shape, "fp64", "advection")
    g_dev = empty(v.shape, "fp64")
    Jd = P.gradient(to_dev(v, "fp64"), g_dev)
    g_host = np.zeros(v.shape)
    Jh = P.gradient(np.ascontiguousarray(v), g_host)
    assert Jd == Jh and np.array_equal(host(g_dev), g_host)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("model", ["advection", "continuity"])
def test_autograd_transport_vjp_matches_oracle_body_force(prec, model):
    import torch

    from paper_2510_08782_gb300.autograd import transport

    shape = (16, 12, 20)
    P, O, v = _setup(shape, prec, model, nt=4)
    vt = to_dev(v, prec).requires_grad_(True)
    mT = transport(vt, P)
    ref_states = O.states(v)
    assert rel_l2(host(mT), ref_states[-1]) < TOL[prec]
    gamma = quantise(random_fourier_field(shape, 1, 3, np.random.default_rng(9))[0], prec)
    (mT * to_dev(gamma, prec)).sum().backward()
    # oracle: the VJP is minus the body force with terminal adjoint value gamma
    from oracle.transport import adjoint_states

    mu = osp.div(v)
    lams = adjoint_states(model, gamma, v, 4, mu=mu)
    ref = np.zeros_like(v)
    for j in range(5):
        wj = 0.5 if j in (0, 4) else 1.0
        if model == "continuity":
            ref -= 0.25 * wj * ref_states[j] * osp.grad(lams[j])
        else:
            ref += 0.25 * wj * lams[j] * osp.grad(ref_states[j])
    assert rel_l2(host(vt.grad), -ref) < TOL[prec] * 3


def test_autograd_incompressible_fd_directions():
    """Config-3 style check at a small size: autograd gradient of the full objective along random
    divergence-free directions vs central finite differences (eps 1e-4) of the FP64 oracle objective,
    to the discretisation error of the optimise-then-discretise gradient."""
    import torch

    from paper_2510_08782_gb300.autograd import transport

    shape = (24, 20, 18)
    P, O, v = _setup(shape, "mixed", "incompressible", nt=8, s=1, alpha=1e-2)
    v = osp.leray(v)
    vt = to_dev(v, "mixed").requires_grad_(True)
    m1 = to_dev(O.m1, "mixed")
    hd = osp.cell_volume(shape)
    loss = 0.5 * hd * ((transport(vt, P) - m1) ** 2).sum()
    loss.backward()
    gdata = host(vt.grad)
    rng = np.random.default_rng(11)
    errs = []
    for _ in range(4):
        d = osp.leray(random_fourier_field(shape, 3, 4, rng))
        d /= np.abs(d).max()
        eps = 1e-4
        Op = OProblem(O.m0, O.m1, nt=8, model="incompressible", reg_order=1, alpha=1e-30)
        fd = (Op.objective(v + eps * d) - Op.objective(v - eps * d)) / (2 * eps)
        an = float(np.sum(gdata * d))
        errs.append(abs(fd - an) / abs(fd))
    assert max(errs) < 0.1, errs
