"""FP64 CPU oracle for the GA-NGMRES transport-optimisation hot path (He & Mang, arXiv 2510.08782).

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously-correct NumPy
restatement of what the method computes, written from the paper (Sec. 2.1-2.3,
Eqs. (1)-(10), Algorithms 1-3, Sec. 3.6-3.7). It exists to check the CUDA library; only the test
suite, the smoke check and the benchmark's CPU-baseline leg may import it. It shares
no code with the CUDA path (which lives in the product package and never imports this).

Modules
  spectral   Fourier grid, symbols |k|^{2s}, spectral derivative/divergence, Leray projector (Sec. 2.2, Sec. 3.6)
  interp     periodic cubic Lagrange (tensor-product) interpolation and its exact transpose (Sec. 2.2 SL scheme)
  transport  RK2 characteristics and semi-Lagrangian state/adjoint steps for the three models (Eqs. (1b), (4), (11b))
  problem    objective (Eq. (1a)), reduced gradient (Eq. (3)), preconditioner (Eq. (9)) per model
  solver     Armijo line search with step memory (Eqs. (6)-(7)), q map (Eq. (10)), NGMRES(w) (Alg. 1),
             AA(w) (Alg. 2), GA-NGMRES(w; sigma, tau) (Alg. 3), dense GMRES for the linear-case pins
  diagnostics  deformation map y = x + h u and det grad y (continuity solve from 1), with a spectral
             det(I + grad(h u)) cross-check route
  dto        discretise-then-optimise gradient of the advection objective: transpose scatter adjoint,
             derivative of the interpolant, chain rule through the RK2 departure points

Readings of passages the paper leaves silent, garbled or ambiguous are stated in each
function's docstring. Parity status: every function is pinned by a CPU test against a
closed form, an invariant, a library routine or brute force (see tests/test_oracle_*.py);
the full nonlinear solve has no printed worked example to pin to (parity unpinned at the
level of whole-solve trajectories; its ingredients are pinned).
"""
