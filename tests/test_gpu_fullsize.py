"""Parity at the benchmark's full size: the 256^3 mass-preserving workload (continuity, n_t = 16, H1,
alpha = 1e-3, checkpoint every 4, FP32 fields) with the kernels and launch configuration bench.py times.

The oracle cannot solve the whole problem at this size in seconds, so it checks outputs it can
compute one by one: departure points, one state step and one adjoint step at sampled voxels
(including voxels on brick edges and the periodic seam), derivatives on sampled grid lines, the full
R2C transform against numpy, and the whole gradient and preconditioner at v = 0, where the gradient
has a closed form."""
import numpy as np
import pytest

from gpu_util import TOL, TOL_GRAD_MIXED, empty, host, quantise, rel_l2, to_dev
from oracle import spectral as osp
from oracle.transport import adjoint_step_at, departure_points_at, state_step_at
from synth.inputs import workload

pytestmark = pytest.mark.gpu

N, NT = 256, 16


@pytest.fixture(scope="module")
def full():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_08782_gb300 import Problem, build

    build.build()
    w = workload("cont3d256")
    m0, m1, v = (quantise(w[k], "mixed") for k in ("m0", "m1", "v_true"))
    P = Problem(to_dev(m0, "mixed"), to_dev(m1, "mixed"), nt=NT, model="continuity", reg_order=1, alpha=1e-3,
                prec="mixed", ckpt_every=4, window=10, sigma=4, tau=2)
    rng = np.random.default_rng(2024)
    rand = np.stack([rng.integers(0, N, size=4000) for _ in range(3)])
    # brick edges (x multiples of 32, y and z multiples of 8) and the periodic seam
    edge = np.array([[0, 0, 0], [255, 255, 255], [7, 8, 31], [8, 7, 32], [0, 255, 128], [255, 0, 224],
                     [16, 120, 255], [248, 247, 0]]).T
    pts = np.concatenate([rand, edge], axis=1)
    yield dict(P=P, m0=m0, m1=m1, v=v, mu=osp.div(v), pts=pts, torch=torch)
    P.close()


def test_departure_points_at_sampled_voxels(full):
    import paper_2510_08782_gb300 as ga

    P, v, pts = full["P"], full["v"], full["pts"]
    xm = empty(v.shape, "mixed")
    xp = empty(v.shape, "mixed")
    ga.ga_op_departure(P.ctx, P.dtype, to_dev(v, "mixed"), xm, xp)
    for out, sign in ((xm, +1), (xp, -1)):
        got = np.stack([host(out[a])[tuple(pts)] for a in range(3)])
        ref = departure_points_at(v, NT, sign, pts) - pts
        assert rel_l2(got, ref) < TOL["mixed"], rel_l2(got, ref)


def test_first_state_step_at_sampled_voxels(full):
    import paper_2510_08782_gb300 as ga

    P, v, pts, m0, mu = full["P"], full["v"], full["pts"], full["m0"], full["mu"]
    states = empty((NT + 1, N, N, N), "mixed")
    ga.ga_op_forward(P.ctx, P.dtype, to_dev(v, "mixed"), states)
    got = host(states[1])[tuple(pts)]
    ref = state_step_at("continuity", m0, mu, departure_points_at(v, NT, +1, pts), pts, NT)
    assert rel_l2(got, ref) < TOL["mixed"], rel_l2(got, ref)
    # the continuity scheme keeps the mass to its discretisation error over all 16 steps
    mass0, mass1 = float(states[0].double().sum()), float(states[NT].double().sum())
    assert abs(mass1 - mass0) < 1e-3 * mass0
    del states
    full["torch"].cuda.empty_cache()


def test_last_adjoint_step_at_sampled_voxels(full):
    import paper_2510_08782_gb300 as ga

    P, v, pts, mu = full["P"], full["v"], full["pts"], full["mu"]
    lam1 = full["m1"] - full["m0"]
    lams = empty((NT + 1, N, N, N), "mixed")
    ga.ga_op_adjoint(P.ctx, P.dtype, to_dev(v, "mixed"), to_dev(lam1, "mixed"), lams)
    got = host(lams[NT - 1])[tuple(pts)]
    ref = adjoint_step_at("continuity", lam1, mu, departure_points_at(v, NT, -1, pts), pts, NT)
    assert rel_l2(got, ref) < TOL["mixed"], rel_l2(got, ref)
    del lams
    full["torch"].cuda.empty_cache()


def test_derivatives_and_divergence_on_sampled_lines(full):
    import paper_2510_08782_gb300 as ga

    P, v, m0, pts = full["P"], full["v"], full["m0"], full["pts"][:, :300]
    rng = np.random.default_rng(7)
    for a in range(3):
        out = empty((N, N, N), "mixed")
        ga.ga_op_deriv(P.ctx, P.dtype, to_dev(m0, "mixed"), a, out)
        o = np.moveaxis(host(out), a, -1).reshape(-1, N)
        f = np.moveaxis(m0, a, -1).reshape(-1, N)
        rows = rng.integers(0, N * N, size=64)
        assert rel_l2(o[rows], osp.line_derivative(f[rows])) < 4 * TOL["mixed"], a
    mu = empty((N, N, N), "mixed")
    ga.ga_op_div(P.ctx, P.dtype, to_dev(v, "mixed"), mu)
    ref = np.zeros(pts.shape[1])
    for a in range(3):
        lines = np.moveaxis(v[a], a, -1)  # line through each voxel along axis a
        other = [pts[b] for b in range(3) if b != a]
        ref += osp.line_derivative(lines[tuple(other)])[np.arange(pts.shape[1]), pts[a]]
    assert rel_l2(host(mu)[tuple(pts)], ref) < 4 * TOL["mixed"]


def test_real_transform_matches_numpy(full):
    import paper_2510_08782_gb300 as ga

    P, m0 = full["P"], full["m0"]
    fh = empty((N, N, N // 2 + 1, 2), "mixed")
    ga.ga_op_fft_r2c(P.ctx, P.dtype, to_dev(m0, "mixed"), fh)
    ref = np.fft.rfftn(m0)
    assert rel_l2(host(fh), np.stack([ref.real, ref.imag], axis=-1)) < TOL["mixed"]


def test_gradient_and_preconditioner_at_zero_velocity(full):
    """At v = 0 every departure point is its own grid point and mu = 0, so pi_j = pi_0 for all j and
    lambda_j = pi_1 - pi_0 (Eq. (11) with the continuity adjoint); the trapezoid weights sum to one,
    hence g = -pi_0 grad(pi_1 - pi_0) and obj = 1/2 h^3 sum (pi_0 - pi_1)^2. This exercises the
    checkpointed forward sweep, the 16 adjoint steps, the 17-point body force and the epilogue."""
    P, m0, m1 = full["P"], full["m0"], full["m1"]
    zero = to_dev(np.zeros((3, N, N, N)), "mixed")
    g = empty((3, N, N, N), "mixed")
    J = P.gradient(zero, g)
    gref = -m0[None] * osp.grad(m1 - m0)
    Jref = 0.5 * osp.cell_volume((N, N, N)) * float(np.sum((m0 - m1) ** 2))
    assert abs(J - Jref) <= 1e-9 * Jref, (J, Jref)
    assert rel_l2(host(g), gref) < TOL_GRAD_MIXED, rel_l2(host(g), gref)
    s = empty((3, N, N, N), "mixed")
    P.precond(g, s)
    sref = -osp.apply_alphaL_inv(gref, 1, 1e-3)
    assert rel_l2(host(s), sref) < TOL_GRAD_MIXED, rel_l2(host(s), sref)
