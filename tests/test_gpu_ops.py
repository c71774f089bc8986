"""GPU parity of every operator of the gradient-evaluation path against the FP64 oracle.

Each test feeds the same seeded inputs (quantised to the context element type) to the CUDA
library through its C ABI and to the oracle, and compares element by element (relative L2).
Grids cover 2D and 3D, radix-2/3/5 lengths, several CTA tiles and ragged tails.
"""
import numpy as np
import pytest

from gpu_util import TOL, empty, host, quantise, rel_l2, to_dev
from oracle import spectral as osp
from oracle.transport import adjoint_states, departure_points, forward_states, grid_index
from synth.inputs import random_fourier_field, random_problem_fields

pytestmark = pytest.mark.gpu

SHAPES = [(32, 24), (16, 12, 20), (8, 256, 250)]
PRECS = ["fp64", "mixed"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_08782_gb300 import build

    build.build()


def _problem(shape, prec, model="advection", nt=4, s=2, alpha=1e-3, seed=0, vox=1.2, ckpt=0):
    from paper_2510_08782_gb300 import Problem

    m0, m1, v = random_problem_fields(shape, seed, model=model, vel_scale_vox=vox)
    m0, m1, v = quantise(m0, prec), quantise(m1, prec), quantise(v, prec)
    P = Problem(to_dev(m0, prec), to_dev(m1, prec), nt=nt, model=model, reg_order=s, alpha=alpha,
                prec=prec, ckpt_every=ckpt)
    return P, m0, m1, v


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", SHAPES)
def test_fft_r2c_and_inverse(shape, prec):
    import paper_2510_08782_gb300 as ga

    P, m0, _, _ = _problem(shape, prec)
    f = quantise(random_fourier_field(shape, 1, max(shape) // 2, np.random.default_rng(1))[0], prec)
    fh = empty(shape[:-1] + (shape[-1] // 2 + 1, 2), prec)
    ga.ga_op_fft_r2c(P.ctx, P.dtype, to_dev(f, prec), fh)
    ref = np.fft.rfftn(f)
    got = host(fh)
    assert rel_l2(got, np.stack([ref.real, ref.imag], axis=-1)) < TOL[prec]
    back = empty(shape, prec)
    ga.ga_op_fft_c2r(P.ctx, P.dtype, fh, back)
    assert rel_l2(host(back), f) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", [(32, 24), (16, 12, 20), (64, 48, 40)])
def test_fft_matches_cufft(shape, prec):
    """Cross-check of the hand-written real FFT against cuFFT (through torch.fft) on the same device
    data; cuFFT serves only as this check."""
    import torch

    import paper_2510_08782_gb300 as ga

    P, _, _, _ = _problem(shape, prec)
    f = quantise(random_fourier_field(shape, 1, max(shape) // 2, np.random.default_rng(4))[0], prec)
    fd = to_dev(f, prec)
    fh = empty(shape[:-1] + (shape[-1] // 2 + 1, 2), prec)
    ga.ga_op_fft_r2c(P.ctx, P.dtype, fd, fh)
    ref = torch.view_as_real(torch.fft.rfftn(fd)).cpu().numpy()
    assert rel_l2(host(fh), ref) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", SHAPES)
def test_spectral_derivative_and_divergence(shape, prec):
    import paper_2510_08782_gb300 as ga

    P, _, _, v = _problem(shape, prec)
    d = len(shape)
    f = quantise(random_fourier_field(shape, 1, 6, np.random.default_rng(2))[0], prec)
    ref = osp.grad(f)
    for a in range(d):
        out = empty(shape, prec)
        ga.ga_op_deriv(P.ctx, P.dtype, to_dev(f, prec), a, out)
        assert rel_l2(host(out), ref[a]) < TOL[prec], a
    mu = empty(shape, prec)
    ga.ga_op_div(P.ctx, P.dtype, to_dev(v, prec), mu)
    assert rel_l2(host(mu), osp.div(v)) < TOL[prec] * 10


LONG_AXES = [(4, 8, 512), (4, 512, 8), (512, 4, 8), (6, 10, 384), (4, 480, 6), (1024, 4, 4)]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", LONG_AXES)
def test_fft_and_derivatives_on_long_axes(shape, prec):
    """Transform lengths beyond the compiled plans (384, 480, 512, 1024) along every axis: R2C/C2R and
    the fused derivative passes against numpy."""
    import paper_2510_08782_gb300 as ga

    P, _, _, _ = _problem(shape, prec)
    f = quantise(random_fourier_field(shape, 1, 9, np.random.default_rng(3))[0], prec)
    fh = empty(shape[:-1] + (shape[-1] // 2 + 1, 2), prec)
    ga.ga_op_fft_r2c(P.ctx, P.dtype, to_dev(f, prec), fh)
    ref = np.fft.rfftn(f)
    assert rel_l2(host(fh), np.stack([ref.real, ref.imag], axis=-1)) < TOL[prec]
    back = empty(shape, prec)
    ga.ga_op_fft_c2r(P.ctx, P.dtype, fh, back)
    assert rel_l2(host(back), f) < TOL[prec]
    gref = osp.grad(f)
    for a in range(3):
        out = empty(shape, prec)
        ga.ga_op_deriv(P.ctx, P.dtype, to_dev(f, prec), a, out)
        assert rel_l2(host(out), gref[a]) < TOL[prec] * 4, (a, rel_l2(host(out), gref[a]))


AXES_256 = [(256, 6, 10), (4, 256, 18), (6, 10, 256), (5, 9, 256)]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", AXES_256)
def test_register_transform_on_256_axes(shape, prec):
    """The register-resident passes of 256-point axes: along the contiguous axis (rows; 45 rows leave
    the last packed pencil without a partner) and along strided axes (columns; partial last tiles of
    the 129 half-spectrum columns), for the 3D real transform and its inverse, for one field
    (ga_op_deriv) and for two time steps at once (the body force)."""
    import paper_2510_08782_gb300 as ga

    P, m0, _, v = _problem(shape, prec, model="advection", nt=4)
    f = quantise(random_fourier_field(shape, 1, 6, np.random.default_rng(4))[0], prec)
    fh = empty(shape[:-1] + (shape[-1] // 2 + 1, 2), prec)
    ga.ga_op_fft_r2c(P.ctx, P.dtype, to_dev(f, prec), fh)
    fref = np.fft.rfftn(f)
    assert rel_l2(host(fh), np.stack([fref.real, fref.imag], axis=-1)) < TOL[prec]
    back = empty(shape, prec)
    ga.ga_op_fft_c2r(P.ctx, P.dtype, fh, back)
    assert rel_l2(host(back), f) < TOL[prec]
    ref = osp.grad(f)
    for a in range(3):
        out = empty(shape, prec)
        ga.ga_op_deriv(P.ctx, P.dtype, to_dev(f, prec), a, out)
        assert rel_l2(host(out), ref[a]) < TOL[prec], (a, rel_l2(host(out), ref[a]))
    lam1 = quantise(random_fourier_field(shape, 1, 4, np.random.default_rng(5))[0], prec)
    b = empty(v.shape, prec)
    ga.ga_op_body_force(P.ctx, P.dtype, to_dev(v, prec), to_dev(lam1, prec), b)
    ms = forward_states("advection", m0, v, 4, mu=osp.div(v))
    ls = adjoint_states("advection", lam1, v, 4, mu=osp.div(v))
    bref = np.zeros_like(v)
    for j in range(5):
        bref += 0.25 * (0.5 if j in (0, 4) else 1.0) * ls[j] * osp.grad(ms[j])
    assert rel_l2(host(b), bref) < TOL[prec] * 3


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("s", [1, 2, 3])
@pytest.mark.parametrize("shape", [(32, 24), (16, 12, 20)])
def test_apply_L_and_leray(shape, prec, s):
    import paper_2510_08782_gb300 as ga

    P, _, _, v = _problem(shape, prec, s=s)
    out = empty(v.shape, prec)
    ga.ga_op_apply_L(P.ctx, P.dtype, to_dev(v, prec), out)
    ref = osp.apply_L(v, s)
    # The FFT rounding (about eps log2 n relative, spread over all modes) is amplified by the
    # symbol: |k|^{2s} at the grid corner against the symbol weight of the smooth input.
    eps = 2.0 ** -53 if prec == "fp64" else 2.0 ** -24
    amp = osp.symbol_L(shape, s).max() * np.linalg.norm(v) / np.linalg.norm(ref)
    tol = max(TOL[prec], 4 * eps * np.log2(max(shape)) * amp)
    assert rel_l2(host(out), ref) < tol
    w = quantise(np.random.default_rng(3).standard_normal(v.shape), prec)
    ga.ga_op_leray(P.ctx, P.dtype, to_dev(w, prec), out)
    assert rel_l2(host(out), osp.leray(w)) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", SHAPES)
def test_departure_points(shape, prec):
    import paper_2510_08782_gb300 as ga

    nt = 4
    P, _, _, v = _problem(shape, prec, nt=nt, vox=2.5)
    xm, xp = empty(v.shape, prec), empty(v.shape, prec)
    ga.ga_op_departure(P.ctx, P.dtype, to_dev(v, prec), xm, xp)
    base = grid_index(shape)
    assert rel_l2(host(xm), departure_points(v, nt, +1) - base) < TOL[prec]
    assert rel_l2(host(xp), departure_points(v, nt, -1) - base) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("model", ["advection", "continuity"])
@pytest.mark.parametrize("shape", SHAPES)
def test_state_and_adjoint_steps(shape, prec, model):
    import paper_2510_08782_gb300 as ga

    nt = 3
    P, m0, _, v = _problem(shape, prec, model=model, nt=nt, vox=1.7)
    states = empty((nt + 1,) + shape, prec)
    ga.ga_op_forward(P.ctx, P.dtype, to_dev(v, prec), states)
    mu = osp.div(v)
    ref = forward_states(model, m0, v, nt, mu=mu)
    got = host(states)
    for j in range(nt + 1):
        assert rel_l2(got[j], ref[j]) < TOL[prec], (j, rel_l2(got[j], ref[j]))
    lam1 = quantise(random_fourier_field(shape, 1, 4, np.random.default_rng(4))[0], prec)
    lams = empty((nt + 1,) + shape, prec)
    ga.ga_op_adjoint(P.ctx, P.dtype, to_dev(v, prec), to_dev(lam1, prec), lams)
    lref = adjoint_states(model, lam1, v, nt, mu=mu)
    got = host(lams)
    for j in range(nt + 1):
        assert rel_l2(got[j], lref[j]) < TOL[prec], (j, rel_l2(got[j], lref[j]))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("model", ["advection", "continuity"])
@pytest.mark.parametrize("ckpt,nt", [(0, 5), (2, 5), (2, 4), (3, 7)])
@pytest.mark.parametrize("shape", [(32, 24), (16, 12, 20)])
def test_body_force(shape, prec, model, ckpt, nt):
    """The trapezoid sum over t_j visits the time steps in pairs sharing one derivative pass; odd and
    even n_t (a single last step), with and without checkpoints (segments split across a pair)."""
    import paper_2510_08782_gb300 as ga
    P, m0, _, v = _problem(shape, prec, model=model, nt=nt, ckpt=ckpt)
    lam1 = quantise(random_fourier_field(shape, 1, 4, np.random.default_rng(5))[0], prec)
    b = empty(v.shape, prec)
    ga.ga_op_body_force(P.ctx, P.dtype, to_dev(v, prec), to_dev(lam1, prec), b)
    mu = osp.div(v)
    ms = forward_states(model, m0, v, nt, mu=mu)
    ls = adjoint_states(model, lam1, v, nt, mu=mu)
    ht = 1.0 / nt
    ref = np.zeros_like(v)
    for j in range(nt + 1):
        wj = 0.5 if j in (0, nt) else 1.0
        if model == "continuity":
            ref -= ht * wj * ms[j] * osp.grad(ls[j])
        else:
            ref += ht * wj * ls[j] * osp.grad(ms[j])
    assert rel_l2(host(b), ref) < TOL[prec] * 3


@pytest.mark.parametrize("prec", PRECS)
def test_dots_and_lsq(prec):
    import paper_2510_08782_gb300 as ga
    from oracle.solver import ngmres_lsq

    P, _, _, _ = _problem((16, 12, 20), prec)
    rng = np.random.default_rng(6)
    vecs = [quantise(rng.standard_normal(3 * 16 * 12 * 20), prec) for _ in range(7)]
    dv = [to_dev(x, prec) for x in vecs]
    out = ga.ga_op_dots(P.ctx, P.dtype, dv[0], dv)
    ref = np.array([float(np.dot(vecs[0], x)) for x in vecs])
    # FP64-accurate even for FP32 data (compensated accumulation of exact products)
    assert np.max(np.abs(out - ref) / np.abs(ref)) < 1e-12
    gq, gw = vecs[0], vecs[1:5]
    c = float(gq @ gq)
    a = np.array([gq @ g for g in gw])
    M = np.array([[gi @ gj for gj in gw] for gi in gw])
    beta = ga.ga_op_lsq(P.ctx, c, a, M)
    np.testing.assert_allclose(beta, ngmres_lsq(gq, gw), rtol=1e-9, atol=1e-12)


def test_dots_and_lsq_at_the_largest_window():
    """w = 62: 64 inner products in one call and the 63-entry least-squares solve (the sizes the paper's
    w = 50 runs need), against exact products and the oracle's lstsq on the explicit differences."""
    import paper_2510_08782_gb300 as ga
    from oracle.solver import ngmres_lsq

    P, _, _, _ = _problem((16, 12, 20), "fp64")
    rng = np.random.default_rng(16)
    vecs = [rng.standard_normal(3 * 16 * 12 * 20) for _ in range(64)]
    out = ga.ga_op_dots(P.ctx, P.dtype, to_dev(vecs[0], "fp64"), [to_dev(x, "fp64") for x in vecs])
    ref = np.array([float(np.dot(vecs[0], x)) for x in vecs])
    assert np.max(np.abs(out - ref) / np.abs(ref)) < 1e-12
    gq, gw = vecs[0], vecs[1:]
    c = float(gq @ gq)
    a = np.array([gq @ g for g in gw])
    M = np.array([[gi @ gj for gj in gw] for gi in gw])
    beta = ga.ga_op_lsq(P.ctx, c, a, M)
    assert beta.shape == (63,)
    np.testing.assert_allclose(beta, ngmres_lsq(gq, gw), rtol=1e-8, atol=1e-11)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("model", ["advection", "continuity"])
@pytest.mark.parametrize("vox,kmax", [(14.0, 3), (3.0, 9)])
def test_steps_beyond_halo_and_rough_velocity(prec, model, vox, kmax):
    """Departure points far outside the staged halo (about 7 cells per step) and rough velocities
    whose columns do not share integer offsets take the slow paths of the tiled FP32 kernel."""
    import paper_2510_08782_gb300 as ga
    from synth.inputs import smooth_velocity

    shape = (24, 40, 36)
    nt = 2
    P, m0, _, _ = _problem(shape, prec, model=model, nt=nt)
    v = quantise(smooth_velocity(shape, kmax, vox, np.random.default_rng(12)), prec)
    states = empty((nt + 1,) + shape, prec)
    ga.ga_op_forward(P.ctx, P.dtype, to_dev(v, prec), states)
    mu = osp.div(v)
    ref = forward_states(model, m0, v, nt, mu=mu)
    for j in range(nt + 1):
        assert rel_l2(host(states)[j], ref[j]) < TOL[prec], j
    lams = empty((nt + 1,) + shape, prec)
    ga.ga_op_adjoint(P.ctx, P.dtype, to_dev(v, prec), to_dev(m0, prec), lams)
    lref = adjoint_states(model, m0, v, nt, mu=mu)
    for j in range(nt + 1):
        assert rel_l2(host(lams)[j], lref[j]) < TOL[prec], j
