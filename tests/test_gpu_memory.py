"""Device memory of a context: the workspace planner against what ga_setup really allocates, and the
allocation-failure path (GA_ERR_NOMEM) produced on the host side, without exhausting the GPU."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_08782_gb300 import build

    build.build()


def _fields(n, seed=0):
    import torch

    rng = np.random.default_rng(seed)
    m0 = torch.from_numpy(rng.uniform(0.5, 1.0, n).astype(np.float32)).cuda()
    return m0, torch.roll(m0, 1, 0).contiguous()


def test_planned_workspace_is_what_setup_allocates():
    import torch

    import paper_2510_08782_gb300 as ga

    n = (128, 128, 128)
    m0, m1 = _fields(n)
    warm = ga.Problem(m0, m1, nt=4, model="continuity", reg_order=1, alpha=1e-3, prec="mixed")
    warm.close()  # kernels, plans and tile choices of this grid are loaded and cached now
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    P = ga.Problem(m0, m1, nt=16, model="continuity", reg_order=1, alpha=1e-3, prec="mixed", ckpt_every=4,
                   window=10)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    planned = ga.ga_workspace_bytes(P.desc, P.opts)
    used = free0 - free1
    P.close()
    assert planned > 40 * 8 * 2 ** 20  # about 60 fields of 8 MiB
    # the allocator rounds every one of the context's ~45 allocations up to its page size
    assert planned <= used <= planned + 64 * 2 * 2 ** 20, (planned, used)


def test_setup_refuses_a_workspace_larger_than_free_memory():
    import torch

    import paper_2510_08782_gb300 as ga
    from paper_2510_08782_gb300 import binding

    d = binding.ProblemDesc()
    d.dim, d.n[0], d.n[1], d.n[2] = 3, 1024, 1024, 1024
    d.nt, d.model, d.reg_order, d.alpha, d.prec, d.ckpt_every = 16, 0, 1, 1e-3, ga.GA_PREC_FP64, 0
    o = binding.SolverOpts()
    o.window, o.sigma, o.tau, o.max_iter, o.rel_tol = 40, 4, 2, 10, 1e-2
    o.armijo_c, o.max_backtracks, o.variant, o.method, o.graphs = 1e-4, 20, 1, 0, 0
    need = ga.ga_workspace_bytes(d, o)
    free0, total = torch.cuda.mem_get_info()
    assert need > total
    # ga_setup compares the planned workspace with the free memory before it reads m0, m1 or allocates
    # anything, so small stand-ins for the 8 GiB fields are never touched
    dummy = np.zeros(8, dtype=np.float64)
    h = ctypes.c_void_p(1)
    st = binding.lib().ga_setup(ctypes.byref(d), ctypes.byref(o), dummy.ctypes.data, dummy.ctypes.data,
                                ga.GA_MEM_HOST, None, ctypes.byref(h))
    assert st == 3  # GA_ERR_NOMEM
    assert h.value is None
    msg = ga.ga_last_error(None)
    assert "bytes" in msg and str(need) in msg
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < 64 * 2 ** 20
    # the device stays usable: a small problem sets up and evaluates
    m0, m1 = _fields((32, 32, 32))
    P = ga.Problem(m0, m1, nt=4, model="advection", reg_order=1, alpha=1e-2, prec="mixed")
    v = torch.zeros((3, 32, 32, 32), dtype=torch.float32, device="cuda")
    assert np.isfinite(P.objective(v))
    P.close()
