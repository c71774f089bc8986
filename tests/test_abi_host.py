"""Host-side checks of the C ABI: the library builds, loads and exports every declared symbol,
and argument validation rejects bad descriptors without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libga():
    from paper_2510_08782_gb300 import build

    build.build()
    from paper_2510_08782_gb300 import binding

    return binding


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"\b(ga_[a-z0-9_]+)\s*\(", text))


def test_every_declared_symbol_is_exported(libga):
    L = libga.lib()
    names = _declared("ga.h") | _declared("ga_ops.h")
    assert len(names) >= 25
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing
    # and the binding wraps each of them under the same name
    import paper_2510_08782_gb300 as pkg

    unwrapped = [n for n in sorted(names) if not hasattr(pkg, n)]
    assert not unwrapped, unwrapped


def test_status_strings(libga):
    assert libga.ga_status_str(0) == "GA_OK"
    assert libga.ga_status_str(5) == "GA_ERR_LINESEARCH"


def _desc(libga, **kw):
    d = libga.ProblemDesc()
    d.dim, d.nt, d.model, d.reg_order, d.alpha, d.prec, d.ckpt_every = 2, 4, 0, 1, 1e-2, 0, 0
    d.n[0], d.n[1] = 16, 16
    for k, v in kw.items():
        if k == "n":
            for i, x in enumerate(v):
                d.n[i] = x
        else:
            setattr(d, k, v)
    o = libga.SolverOpts()
    o.window, o.sigma, o.tau, o.max_iter, o.rel_tol = 5, 4, 2, 10, 1e-2
    o.armijo_c, o.max_backtracks, o.variant, o.method = 1e-4, 20, 1, 0
    return d, o


@pytest.mark.parametrize("bad", [dict(dim=4), dict(n=(16, 14)), dict(n=(7, 16)), dict(nt=0),
                                 dict(model=3), dict(reg_order=4), dict(alpha=-1.0), dict(prec=2),
                                 dict(ckpt_every=-1), dict(n=(2048, 16))])
def test_setup_rejects_bad_descriptors(libga, bad):
    d, o = _desc(libga, **bad)
    m = np.zeros((16, 16))
    h = ctypes.c_void_p()
    st = libga.lib().ga_setup(ctypes.byref(d), ctypes.byref(o), m.ctypes.data, m.ctypes.data, 0, None,
                              ctypes.byref(h))
    assert st == 1 and not h.value
    assert "invalid" in libga.ga_last_error(None)


@pytest.mark.parametrize("bad", [dict(window=63), dict(sigma=0), dict(tau=-1), dict(max_iter=0),
                                 dict(variant=3), dict(armijo_c=0.0), dict(method=5), dict(graphs=3),
                                 dict(graphs=2, method=2)])
def test_setup_rejects_bad_options(libga, bad):
    d, o = _desc(libga)
    for k, v in bad.items():
        setattr(o, k, v)
    m = np.zeros((16, 16))
    h = ctypes.c_void_p()
    st = libga.lib().ga_setup(ctypes.byref(d), ctypes.byref(o), m.ctypes.data, m.ctypes.data, 0, None,
                              ctypes.byref(h))
    assert st == 1


def test_null_arguments_rejected(libga):
    L = libga.lib()
    out = ctypes.c_double()
    assert L.ga_objective(None, None, 0, ctypes.byref(out)) == 1
    assert L.ga_gradient(None, None, None, 0, None) == 1
    assert L.ga_step(None, None, 0, None) == 1
    assert L.ga_deformation(None, None, None, None, 0) == 1
    assert L.ga_gradient_dto(None, None, None, 0, None) == 1
    assert L.ga_transport_vjp_exact(None, None, None, None, 0) == 1
    assert L.ga_solve_batch(-1, None, None, 0, None) == 1
    assert L.ga_setup(None, None, None, None, 0, None, None) == 1
    tiles = (ctypes.c_int * 6)()
    assert L.ga_op_get_tiles(None, tiles) == 1
    assert L.ga_op_set_tiles(None, tiles) == 1
    assert L.ga_prof_start(None, 4) == 1
    assert L.ga_get_stats(None, None) == 1


def test_binding_rejects_unknown_graph_mode(libga):
    """Problem() checks its graph mode before it touches the device."""
    from paper_2510_08782_gb300 import Problem

    m = np.zeros((16, 16))
    with pytest.raises(ValueError):
        Problem(m, m, nt=2, graphs="sometimes")


def test_binding_rejects_wrong_dtype(libga):
    from paper_2510_08782_gb300.binding import GaError, _ptr

    with pytest.raises(GaError):
        _ptr(np.zeros(4, dtype=np.float32), np.float64)
    with pytest.raises(GaError):
        _ptr(np.zeros((4, 4))[:, ::2], np.float64)


def test_binding_rejects_arrays_that_do_not_match_the_context_grid(libga):
    """The C calls read and write as many elements as the context's grid implies; the binding refuses
    a short or long array (or a short pointer list or output for the inner products) before any call
    reaches the library."""
    b = libga
    fake = 0x1234  # a registered grid only: every check below raises before the C call
    b._CTX_INFO[fake] = (3, (4, 6, 8), 2, None)
    try:
        n = 4 * 6 * 8
        vec, short = np.zeros(3 * n, np.float32), np.zeros(3 * n - 1, np.float32)
        with pytest.raises(b.GaError, match="elements"):
            b.ga_op_departure(fake, np.float32, vec, short, vec)
        with pytest.raises(b.GaError, match="elements"):
            b.ga_op_forward(fake, np.float32, vec, np.zeros(2 * n, np.float32))  # needs (n_t + 1) n
        with pytest.raises(b.GaError, match="elements"):
            b.ga_op_fft_r2c(fake, np.float32, np.zeros(n, np.float32), np.zeros(n, np.float32))
        with pytest.raises(b.GaError, match="elements"):
            b.ga_gradient(fake, np.float32, vec, short)
        with pytest.raises(b.GaError, match="b\\[1\\]"):
            b.ga_op_dots(fake, np.float32, vec, [vec, short])
    finally:
        b._CTX_INFO.pop(fake, None)
    with pytest.raises(b.GaError, match="b\\[0\\]"):
        b.ga_dots_noalloc(np.float32, np.zeros(8, np.float32), [np.zeros(7, np.float32)], np.zeros(1))


def _desc_opts(libga, n=(16, 16, 16), prec=1, nt=16, K=0, window=5, graphs=0):
    d = libga.ProblemDesc()
    d.dim = len(n)
    for i, x in enumerate(n):
        d.n[i] = x
    d.nt, d.model, d.reg_order, d.alpha, d.prec, d.ckpt_every = nt, 1, 1, 1e-3, prec, K
    o = libga.SolverOpts()
    o.window, o.sigma, o.tau, o.max_iter, o.rel_tol = window, 4, 2, 10, 1e-2
    o.armijo_c, o.max_backtracks, o.variant, o.method, o.graphs = 1e-4, 20, 1, 0, graphs
    return d, o


def test_workspace_planner_follows_the_context_layout(libga):
    """ga_workspace_bytes is host arithmetic: each part of the context layout changes it by the
    bytes that part holds."""
    wb = libga.ga_workspace_bytes
    n = (16, 16, 16)
    nv, s = 16 ** 3, 4
    vl = 3 * nv
    base = wb(*_desc_opts(libga, n))
    # one more window slot: one more iterate (v and alpha L v) and gradient, and a larger FP64 Gram
    w6 = wb(*_desc_opts(libga, n, window=6))
    assert w6 - base == 3 * vl * s + (7 * 7 - 6 * 6) * 8
    # checkpoints every 4 of 16 steps: 4 stored states and two segment buffers of 3 recomputed states
    # instead of 16 states
    ck = wb(*_desc_opts(libga, n, K=4))
    assert base - ck == (16 - 4 - 2 * 3) * nv * s
    # FP64 doubles every field; the FP64 scratch arrays and the Gram do not change
    d64 = wb(*_desc_opts(libga, n, prec=0))
    fixed = base - (d64 - base)
    assert 0 < fixed < 1_000_000
    # an invalid descriptor is refused like ga_setup refuses it
    with pytest.raises(libga.GaError):
        wb(*_desc_opts(libga, (16, 16, 7)))
