"""ga_dots_noalloc: the inner products for callers that cannot allocate device memory.

A program that has handed all of its device memory to its own allocator or pool, or a
latency-critical loop that must not pay for cudaMalloc/cudaFree, cannot create a context (ga_setup
allocates). ga_dots_noalloc serves such callers: it keeps its per-CTA partial sums in a fixed device
array inside the library. These tests call it through the C ABI twice in a row and compare each
result with the context-based ga_op_dots, for FP64 and FP32 data, and check that a request larger
than the fixed array is refused. This file is collected last on purpose, so that a failure here does
not hide the rest of the suite; it also passes when run on its own in a fresh process.
"""
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


@pytest.mark.parametrize("count", [1, 6, 17, 32])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_dots_match_context_dots_on_two_calls(prec, count):
    import torch

    import paper_2510_08782_gb300 as ga
    from paper_2510_08782_gb300 import binding

    dtype = np.float64 if prec == "fp64" else np.float32
    tdtype = torch.float64 if prec == "fp64" else torch.float32
    shape = (16, 12, 20)
    rng = np.random.default_rng(31)
    m0 = torch.from_numpy(rng.uniform(0.5, 1.0, shape).astype(dtype)).cuda()
    P = ga.Problem(m0, m0.clone(), nt=2, model="advection", reg_order=1, alpha=1e-2, prec=prec)
    L = binding.lib()
    code = ga.GA_PREC_FP64 if prec == "fp64" else ga.GA_PREC_MIXED
    n = 3 * int(np.prod(shape))
    for _ in range(2):  # two calls in a row: the fixed scratch array keeps the previous call's data
        host = [rng.standard_normal(n).astype(dtype) for _ in range(count)]
        vecs = [torch.from_numpy(x).cuda() for x in host]
        a = vecs[0]
        ref = ga.ga_op_dots(P.ctx, P.dtype, a, vecs)
        out = torch.full((count,), float("nan"), dtype=torch.float64, device="cuda")
        ptrs = (ctypes.c_void_p * count)(*[v.data_ptr() for v in vecs])
        st = L.ga_dots_noalloc(code, a.data_ptr(), ptrs, count, n, out.data_ptr(), None)
        assert st == 0, ga.ga_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0.0)
        # and directly against the products summed in FP64 on the host: the inputs are exact in FP64,
        # so both sides carry only summation error (compensated on the device, pairwise in NumPy)
        a64 = host[0].astype(np.float64)
        for i, x in enumerate(host):
            prods = a64 * x.astype(np.float64)
            assert abs(got[i] - prods.sum()) <= 64 * 2.3e-16 * np.abs(prods).sum(), i


def test_noalloc_dots_refuse_more_vectors_than_the_fixed_array_holds():
    import torch

    import paper_2510_08782_gb300 as ga
    from paper_2510_08782_gb300 import binding

    a = torch.ones(64, dtype=torch.float64, device="cuda")
    out = torch.zeros(33, dtype=torch.float64, device="cuda")
    ptrs = (ctypes.c_void_p * 33)(*([a.data_ptr()] * 33))
    st = binding.lib().ga_dots_noalloc(ga.GA_PREC_FP64, a.data_ptr(), ptrs, 33, 64, out.data_ptr(), None)
    assert st == 1
    assert "32" in ga.ga_last_error(None)
