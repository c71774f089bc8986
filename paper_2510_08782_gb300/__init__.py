"""GB300 (sm_103a) library for GA-NGMRES-accelerated transport-constrained optimisation.

He & Mang, "A generalized alternating NGMRES method for PDE-constrained optimization problems
governed by transport equations" (arXiv 2510.08782). The compute path is the CUDA library
libga_gb300.so (C ABI in include/ga.h and include/ga_ops.h); this package is a thin ctypes binding
with the same function names plus a torch.autograd wrapper. It has no CPU fallback: importing a
function raises if the library is missing, and every call runs the library's kernels.
"""
from .binding import (  # noqa: F401
    GA_MEM_DEVICE,
    GA_MEM_HOST,
    GA_METHOD_GA_NGMRES,
    GA_METHOD_RPGD,
    GA_MODEL_ADVECTION,
    GA_MODEL_CONTINUITY,
    GA_MODEL_INCOMPRESSIBLE,
    GA_PREC_FP64,
    GA_PREC_MIXED,
    GaError,
    Problem,
    ProblemDesc,
    SolverOpts,
    Stats,
    STATUS,
    ga_destroy,
    ga_gradient,
    ga_last_error,
    ga_objective,
    ga_op_adjoint,
    ga_op_apply_L,
    ga_op_body_force,
    ga_op_departure,
    ga_op_deriv,
    ga_op_div,
    ga_op_dots,
    ga_op_fft_c2r,
    ga_op_fft_r2c,
    ga_op_forward,
    ga_op_leray,
    ga_op_lsq,
    ga_precond,
    ga_prof_start,
    ga_prof_stop,
    ga_reset,
    ga_setup,
    ga_solve,
    ga_solve_batch,
    ga_status_str,
    ga_step,
    ga_transport,
    ga_transport_vjp,
    lib,
    library_path,
)
