"""Shared helpers of the GPU parity tests (CUDA library vs FP64 oracle)."""
import numpy as np

# Tolerances on relative L2 error against the FP64 oracle.
TOL = {
    "fp64": 1e-10,      # every FP64 kernel
    "mixed": 1e-5,      # FP32 transport, FFT and spectral kernels
}
# Whole-gradient evaluations in mixed precision chain n_t FP32 transport steps, FP32 FFT-derivative
# passes and an FP32 spectral epilogue; the FP32 rounding of each stage (about 6e-8 relative)
# accumulates over O(n_t) stages and the mismatch m1 - m(1) cancels leading digits, so the bar for a
# full mixed gradient is looser than for one kernel.
TOL_GRAD_MIXED = 2e-4


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0))


def dtype_of(prec):
    return np.float64 if prec == "fp64" else np.float32


def to_dev(x, prec):
    import torch

    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, dtype=dtype_of(prec)))).cuda()


def empty(shape, prec):
    import torch

    return torch.empty(tuple(shape), dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def quantise(x, prec):
    """The inputs exactly as the GPU sees them (cast to the element type), back in float64."""
    return np.asarray(x, dtype=dtype_of(prec)).astype(np.float64)
