// Internal launchers of the GB300 GA-NGMRES library. Every launcher enqueues work on `st`
// and returns cudaGetLastError() of its launch(es).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace ga {

constexpr int kThreads = 256;       // threads per CTA of the streaming kernels
constexpr int kRedBlocks = 152 * 4; // CTAs of the reduction kernels (4 per SM of a GB300)
constexpr int kMaxDots = 64;        // vectors per multi-dot call
constexpr int kMaxWin = 63;         // window entries in the least-squares kernel
constexpr int kSlDepths[3] = {8, 4, 12};  // brick depths of the FP32 3D transport steps (Grid::sl_bz, sl_bz_adj)
constexpr int kRegFftLen = 256;      // axis length of the register-resident derivative passes
constexpr int kRegFftPencils = 16;   // complex pencils per CTA of those passes

template <typename T> struct PtrList { const T* p[16]; };

// Counts kernel launches issued by the library (process-wide).
void note_launches(int n);
// Message returned by ga_last_error(NULL) on this thread (calls that have no context).
void set_global_error(const char* msg);

template <typename T> struct FftTables {
  FftPlan plan[3];
  const cx<T>* tw[3];  // device tables exp(-2 pi i m / n_a), m < n_a
  // pencils per CTA of the derivative pass along each internal axis (0: deriv_default_pencils); the
  // tile holds 2 B real pencils. Chosen per context by timing; no result depends on it.
  int deriv_pencils[3] = {0, 0, 0};
  int pair_pencils[3] = {0, 0, 0};  // the same for the two-time-step passes of the body force
};

// ---- spectral / FFT passes (fft_kernels.cu) --------------------------------------------------
// out (+)= coef * mult * d f / d x_axis (1D spectral derivative along internal axis `axis`).
template <typename T>
cudaError_t launch_deriv(const Grid& g, const FftTables<T>& ft, int axis, const T* f, const T* mult,
                         T* out, T coef, bool accumulate, cudaStream_t st);
// Two time steps of the body force in one pass: out (+)= coef mult d f + coef2 mult2 d f2 along
// internal axis `axis`, formed as two successive launch_deriv calls would form it (mult, mult2 may be
// null for 1). f and f2 share each complex FFT (real and imaginary parts).
template <typename T>
cudaError_t launch_deriv_pair(const Grid& g, const FftTables<T>& ft, int axis, const T* f, const T* mult, T coef,
                              const T* f2, const T* mult2, T coef2, T* out, bool accumulate, cudaStream_t st);
// Default pencils per CTA of a derivative pass of length L, and whether B pencils fit in one CTA's
// shared memory on this device.
template <typename T> int deriv_default_pencils(int L);
template <typename T> bool deriv_pencils_fit(int L, int B);
// Forward real-to-complex 3D (or 2D) FFT, unnormalised; fh: nhalf complex.
template <typename T>
cudaError_t launch_r2c(const Grid& g, const FftTables<T>& ft, const T* f, cx<T>* fh, cudaStream_t st);
// Inverse (normalised by 1/nvox); overwrites fh.
template <typename T>
cudaError_t launch_c2r(const Grid& g, const FftTables<T>& ft, cx<T>* fh, T* f, cudaStream_t st);

// ---- pointwise spectral operators (spectral_kernels.cu) --------------------------------------
enum SpecMode { SPEC_APPLY_L = 0, SPEC_LERAY = 1, SPEC_PRECOND = 2, SPEC_APPLY_ALPHA_L = 3 };
struct SpecArgs {
  int mode;
  int s;            // regulariser order
  double alpha;
  int project;      // PRECOND: apply the Leray projector first (incompressible model)
};
// x[c] (dim half spectra) updated in place.
template <typename T>
cudaError_t launch_spectral(const Grid& g, const SpecArgs& a, cx<T>* x, cudaStream_t st);
// t = -(g - mean(g)) per component (= alpha L s for s = -(alpha L)^{-1} g), the means taken from the
// zero modes of gh, the half spectrum of g
template <typename T>
cudaError_t launch_neg_centered(const Grid& g, const T* gv, const cx<T>* gh, T* t, cudaStream_t st);

// ---- semi-Lagrangian transport (sl_kernels.cu) -----------------------------------------------
// Displacements (grid units) of the RK2 departure points X- (xm) and, when both != 0, X+ (xp).
template <typename T>
cudaError_t launch_departure(const Grid& g, const T* v, T* xm, T* xp, T ht, cudaStream_t st, int both = 1);
cudaError_t launch_departure_tile(const Grid& g, const float* v, float* xm, float* xp, float ht, int both,
                                  cudaStream_t st);
// One state step m_{j+1} = I[m_j](X-) (continuity: with the RK2 source of -pi div v). For the two-field
// steps of FP32 3D grids (continuity state, advection adjoint), qout (optional) receives the pairs
// (m_{j+1}, m_{j+1} mu) of the output, and qin (optional) gives the same pairs of the input, which the
// step then stages as they are instead of m and mu.
template <typename T>
cudaError_t launch_sl_forward(const Grid& g, int continuity, const T* m, const T* xm, const T* mu,
                              T* out, T ht, cudaStream_t st, const cx<T>* qin = nullptr, cx<T>* qout = nullptr);
// Tiled FP32 3D state (adjoint = 0) or adjoint (adjoint = 1) step (sl_tile_kernels.cu).
cudaError_t launch_sl_tile(const Grid& g, int adjoint, int continuity, const float* f, const float* disp,
                           const float* mu, float* out, float ht, cudaStream_t st, const float2* qin = nullptr,
                           float2* qout = nullptr);
// One adjoint step lambda_j from lambda_{j+1} (advection: with the source lambda div v).
template <typename T>
cudaError_t launch_sl_adjoint(const Grid& g, int continuity, const T* lam, const T* xp, const T* mu,
                              T* out, T ht, cudaStream_t st, const cx<T>* qin = nullptr, cx<T>* qout = nullptr);

// ---- reductions and vector kernels (reduce_kernels.cu) ---------------------------------------
// out[i] = sum_j a[j] b_i[j] for i < count (count <= 32), FP64 compensated; out is device memory.
template <typename T>
cudaError_t launch_dots(const T* a, const T* const* b, int count, long long len, double* partial,
                        double* out, cudaStream_t st);
template <typename T>
cudaError_t launch_maxabs(const T* x, long long len, double* partial, double* out, cudaStream_t st);
// lam = m1 - mT and out[0] = sum (mT - m1)^2.
template <typename T>
cudaError_t launch_mismatch(const T* mT, const T* m1, T* lam, long long len, double* partial,
                            double* out, cudaStream_t st);
cudaError_t launch_sum_partials(const double* partial, int count, int nblocks, double* out, cudaStream_t st);
// discretise-then-optimise sweep (dto_kernels.cu)
template <typename T>
cudaError_t launch_dto_accum(const Grid& g, const T* r, const T* m, const T* disp, T* G, T coef, cudaStream_t st);
template <typename T>
cudaError_t launch_interp_scatter(const Grid& g, const T* r, const T* disp, T* out, cudaStream_t st);
template <typename T>
cudaError_t launch_dto_velocity(const Grid& g, const T* v, const T* G, T* out, T ht, cudaStream_t st);
template <typename T>
cudaError_t launch_fill(T* y, double value, long long len, cudaStream_t st);
// y = x + a s
template <typename T>
cudaError_t launch_axpy(T* y, const T* x, const T* s, double a, long long len, cudaStream_t st);
// out = q + sum_i beta_i (q - v_i), beta on the device
template <typename T>
cudaError_t launch_combine(T* out, const T* q, const T* const* v, const double* beta, int m, long long len,
                           cudaStream_t st);
// NGMRES least squares from FP64 Gram data on the device (single CTA):
// dots[0] = c, dots[1 + i] = a_i, M (m x m, leading dim ldm) -> beta[0..m)
cudaError_t launch_lsq(int m, const double* dots, const double* M, int ldm, double* beta, double* info,
                       cudaStream_t st);
// Window Gram update: M' = [[row0, row[1..]], [row[1..]^T, M[:mkeep, :mkeep]]]
cudaError_t launch_gram_push(double* M, int ldm, int mkeep, const double* row, cudaStream_t st);

// ---- device-driven solve (control_kernels.cu, and ring variants in reduce_kernels.cu) ---------
// The scalars of one problem's iteration (Alg. 3, or RPGD, with the Armijo line search of
// Eqs. (6)-(7)) kept in device memory, so that a whole solve runs as one CUDA graph: small control
// kernels update them and set the graph's conditional nodes (iteration loop, line-search loop, step
// kind). The window of (v, g) pairs is a ring of W1 slots in device memory; entry i (0 = newest) is
// slot (head - i) mod W1 and holds m entries.
struct ResCtl {
  // parameters, written by the host before a launch
  double armijo_c, rel_tol, hd;
  int max_backtracks, kmax, stop_on_converged, sigma, tau, variant, method, W1;
  // iteration state
  int started, k, m, head, trial, branch, last_branch, status;
  int converged, fp_steps;
  double J, mis, Jn, misn, g0inf, ginf, rel_grad_inf, rho, rho_mem, last_rho, gs;
  long long grad_evals, obj_evals, ls_trials, pde_solves;
};
// Status values written to ResCtl::status (those of ga_status).
constexpr int kResErrNan = 4;
constexpr int kResErrLinesearch = 5;
// Which gradient evaluation just finished (launch_res_grad).
enum ResGrad { RES_GRAD_START = 0, RES_GRAD_ACCEPTED = 1, RES_GRAD_TRIAL = 2, RES_GRAD_COMBINED = 3 };

// h_start = !started
cudaError_t launch_res_enter(ResCtl* c, cudaGraphConditionalHandle h_start, cudaStream_t st);
// Bookkeeping after a gradient evaluation whose results are res[0] = sum (m(1) - m1)^2,
// res[1] = sum v . alpha L v, res[2] = ||g||_inf.
cudaError_t launch_res_grad(ResCtl* c, const double* res, int which, cudaStream_t st);
// After a window push: head and m advance; with `iteration`, k advances, the accepted objective becomes
// the current one, the stop test is taken and h_iter is set for the next iteration.
cudaError_t launch_res_pushed(ResCtl* c, int iteration, cudaGraphConditionalHandle h_iter, cudaStream_t st);
// h_iter = (iteration k may run)
cudaError_t launch_res_loop_cond(ResCtl* c, cudaGraphConditionalHandle h_iter, cudaStream_t st);
// Line search start: gs = h^d * gs_raw[0], rho = rho_mem, h_ls = 1.
cudaError_t launch_res_ls_begin(ResCtl* c, const double* gs_raw, cudaGraphConditionalHandle h_ls, cudaStream_t st);
// Armijo test of the trial whose objective sums are res[0..1]; h_ls = (another trial follows).
cudaError_t launch_res_ls_check(ResCtl* c, const double* res, cudaGraphConditionalHandle h_ls, cudaStream_t st);
// h_sw = 0 (fixed-point step), 1 (NGMRES step) or 2 (failed: no step) for iteration k.
cudaError_t launch_res_branch(ResCtl* c, cudaGraphConditionalHandle h_sw, cudaStream_t st);
// y = x + rho s with rho = *a read on the device
template <typename T>
cudaError_t launch_axpy_dev(T* y, const T* x, const T* s, const double* a, long long len, cudaStream_t st);
// out[0] = <a, first>, out[1 + i] = <a, ring entry i> for i < n, n = m (keep = 0) or min(m, W1 - 1)
// (keep = 1); the same compensated sums as launch_dots.
template <typename T>
cudaError_t launch_dots_ring(const T* a, const T* first, const T* ring, long long stride, const ResCtl* c, int W1,
                             int keep, long long len, double* partial, double* out, cudaStream_t st);
// out = q + sum_{i < m} beta_i (q - ring entry i), as launch_combine
template <typename T>
cudaError_t launch_combine_ring(T* out, const T* q, const T* ring, long long stride, const ResCtl* c, int W1,
                                const double* beta, long long len, cudaStream_t st);
// ring slot (head + 1) mod W1 = src (skipped once status != 0)
template <typename T>
cudaError_t launch_ring_store(T* ring, long long stride, const ResCtl* c, int W1, const T* src, long long len,
                              cudaStream_t st);
// launch_lsq and launch_gram_push with m and the kept count read from c (skipped once status != 0)
cudaError_t launch_lsq_ring(const ResCtl* c, int W1, const double* dots, const double* M, double* beta, double* info,
                            cudaStream_t st);
cudaError_t launch_gram_push_ring(double* M, int W1, const ResCtl* c, const double* row, cudaStream_t st);

}  // namespace ga
