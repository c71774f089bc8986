"""The tile autotuner of the FFT-derivative passes: ga_setup times candidate tile shapes (pencils per
CTA) on the context's grid and keeps the fastest. Every pencil is transformed on its own, so each
candidate must give bit-identical derivatives, body forces and gradients."""
import numpy as np
import pytest

from gpu_util import empty, host, to_dev
from synth.inputs import random_problem_fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_08782_gb300 import build

    build.build()


def _problem(shape, prec, model="advection"):
    from paper_2510_08782_gb300 import Problem

    m0, m1, v = random_problem_fields(shape, 7, model=model, vel_scale_vox=1.1)
    dt = np.float64 if prec == "fp64" else np.float32
    P = Problem(to_dev(m0.astype(dt), prec), to_dev(m1.astype(dt), prec), nt=3, model=model, reg_order=1,
                alpha=1e-2, prec=prec)
    return P, v.astype(dt), m0.astype(dt)


@pytest.mark.parametrize("shape,prec", [((40, 48, 64), "mixed"), ((24, 30, 36), "fp64"), ((96, 80), "mixed")])
def test_every_tile_candidate_gives_identical_results(shape, prec):
    from paper_2510_08782_gb300 import ga_op_body_force, ga_op_deriv, ga_op_get_tiles, ga_op_set_tiles

    P, v, m0 = _problem(shape, prec)
    dim = len(shape)
    tuned = ga_op_get_tiles(P.ctx, dim)
    ga_op_set_tiles(P.ctx, [0] * (2 * dim))
    default = ga_op_get_tiles(P.ctx, dim)
    for t, d in zip(tuned, default):
        assert t in (d, max(d // 2, 1), 2 * d), (tuned, default)

    f = to_dev(m0, prec)
    vd = to_dev(v, prec)
    lam1 = to_dev(np.random.default_rng(1).standard_normal(shape), prec)

    def run():
        outs = []
        for a in range(dim):
            df = empty(shape, prec)
            ga_op_deriv(P.ctx, P.dtype, f, a, df)
            outs.append(host(df))
        b = empty((dim,) + shape, prec)
        ga_op_body_force(P.ctx, P.dtype, vd, lam1, b)
        outs.append(host(b))
        g = empty((dim,) + shape, prec)
        outs.append(np.array([P.gradient(vd, g)]))
        outs.append(host(g))
        return outs

    ref = run()
    for k in range(3):
        for a in range(2 * dim):  # one-field passes, then the body force's two-time-step passes
            tiles = list(default)
            tiles[a] = [default[a], max(default[a] // 2, 1), 2 * default[a]][k]
            try:
                ga_op_set_tiles(P.ctx, tiles)
            except Exception:  # a doubled tile that does not fit in shared memory is refused
                continue
            assert ga_op_get_tiles(P.ctx, dim) == tiles
            for x, y in zip(run(), ref):
                assert np.array_equal(x, y)


def test_set_tiles_rejects_bad_shapes():
    from paper_2510_08782_gb300 import GaError, ga_op_get_tiles, ga_op_set_tiles

    P, _, _ = _problem((32, 32, 32), "mixed")
    before = ga_op_get_tiles(P.ctx, 3)
    assert len(before) == 6
    for bad in ([-1, 0, 0, 0, 0, 0], [0, 4096, 0, 0, 0, 0], [0, 0, 0, 0, 0, -2]):
        with pytest.raises(GaError) as e:
            ga_op_set_tiles(P.ctx, bad)
        assert e.value.status == 1
    assert ga_op_get_tiles(P.ctx, 3) == before


@pytest.mark.parametrize("model", ["continuity", "advection"])
@pytest.mark.parametrize("shape", [(40, 48, 64), (30, 16, 40)])
def test_every_brick_depth_gives_identical_transport(shape, model):
    """The brick depths of the FP32 3D state and adjoint steps (z voxels per thread) are chosen at setup by
    timing; every combination gives bit-identical states, adjoint states and gradients, including a
    ragged last brick along z (30 is no multiple of 4, 8 or 12)."""
    from paper_2510_08782_gb300 import GaError, ga_op_adjoint, ga_op_forward, ga_op_get_sl_depth, ga_op_set_sl_depth

    P, v, m0 = _problem(shape, "mixed", model=model)
    sd, ad = ga_op_get_sl_depth(P.ctx)
    assert sd in (4, 8, 12) and ad in (4, 8, 12)
    vd = to_dev(v, "mixed")
    lam1 = to_dev(np.random.default_rng(2).standard_normal(shape), "mixed")

    def run():
        st = empty((4,) + shape, "mixed")
        ga_op_forward(P.ctx, P.dtype, vd, st)
        la = empty((4,) + shape, "mixed")
        ga_op_adjoint(P.ctx, P.dtype, vd, lam1, la)
        g = empty((3,) + shape, "mixed")
        obj = P.gradient(vd, g)
        return [host(st), host(la), host(g), np.array([obj])]

    outs = {}
    for depths in ((4, 4), (8, 8), (12, 12), (12, 4), (4, 12)):  # (state steps, adjoint steps)
        ga_op_set_sl_depth(P.ctx, *depths)
        assert ga_op_get_sl_depth(P.ctx) == depths
        outs[depths] = run()
    for depths, out in outs.items():
        for x, y in zip(out, outs[(8, 8)]):
            assert np.array_equal(x, y), depths
    for bad in ((5, 8), (8, 16)):
        with pytest.raises(GaError) as e:
            ga_op_set_sl_depth(P.ctx, *bad)
        assert e.value.status == 1
    ga_op_set_sl_depth(P.ctx, 0, 0)
    assert ga_op_get_sl_depth(P.ctx) == (8, 8)
