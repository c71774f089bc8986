/*
 * ga_ops.h - operator-level entry points of the GB300 GA-NGMRES library.
 *
 * Each call runs one step of the gradient-evaluation hot path on DEVICE buffers of a context
 * created by ga_setup (include/ga.h), in the context's element type (double for GA_PREC_FP64,
 * float for GA_PREC_MIXED) and layout (scalar field: prod(n) elements, C order; vector field:
 * dim scalar fields back to back). They are ordered on the context stream and return once the
 * result is complete. Buffers are borrowed for the call; outputs must not alias inputs unless
 * stated. Status codes and ga_last_error() behave as in ga.h. These are the building blocks the
 * solver calls; they are exported so that each step can be checked and composed on its own
 * (the torch.autograd wrapper uses ga_transport / ga_transport_vjp).
 */
#ifndef GA_OPS_H
#define GA_OPS_H

#include <stddef.h>
#include "ga.h"

#ifdef __cplusplus
extern "C" {
#endif

/* RK2 departure points of the semi-Lagrangian scheme (Sec. 2.2), as displacements in grid units:
 * X-(x) = x - (h_t/2)(v(x) + v(x - h_t v(x))) for the state equation, X+ the same with -v for
 * the adjoint. xm, xp: dim scalar fields each (component c = displacement along axis c / h_c). */
ga_status ga_op_departure(ga_ctx* ctx, const void* v, void* xm, void* xp);

/* All states m_0..m_{n_t} of the state equation (Eq. (1b) or (11b)) for velocity v.
 * states: (n_t + 1) scalar fields. */
ga_status ga_op_forward(ga_ctx* ctx, const void* v, void* states);

/* All adjoint states lambda_0..lambda_{n_t} (Eq. (4); continuity model: pure backward
 * advection) from the terminal value lam1. lams: (n_t + 1) scalar fields. */
ga_status ga_op_adjoint(ga_ctx* ctx, const void* v, const void* lam1, void* lams);

/* Body force of the reduced gradient (Eq. (3)), trapezoidal in time (Sec. 2.2):
 * b = h_t sum_j w_j lambda_j grad m_j (continuity: b = -h_t sum_j w_j pi_j grad lambda_j), with
 * the states of v and the adjoint started from lam1. No projection. b: vector field. */
ga_status ga_op_body_force(ga_ctx* ctx, const void* v, const void* lam1, void* b);

/* Spectral derivative along one axis (Sec. 2.2): df = F^{-1}[i k~_axis F f], k~ zero at Nyquist. */
ga_status ga_op_deriv(ga_ctx* ctx, const void* f, int axis, void* df);

/* Tile shapes of the context's FFT-derivative passes: the number of complex pencils one CTA
 * transforms. pencils[c] (c = 0..dim-1, the descriptor's axis order) is for the one-field passes
 * along axis c (divergence, ga_op_deriv); pencils[dim + c] for the body force's passes that take two
 * time steps at once. ga_setup picks each by timing the default, its half and its double on the
 * context's own grid (cached per precision and grid for the process). No result depends on them.
 * ga_op_set_tiles overrides them: a value of 0 restores the library default; GA_ERR_ARG if a value is
 * negative or does not fit in one CTA's shared memory. A 256-point axis uses a register-resident
 * transform of 16 complex pencils per CTA: it reports 16 and ignores a set value. CUDA graphs the context recorded earlier keep
 * the shapes they were recorded with. pencils: HOST array of 2 * dim ints. */
ga_status ga_op_get_tiles(const ga_ctx* ctx, int* pencils);
ga_status ga_op_set_tiles(ga_ctx* ctx, const int* pencils);

/* Brick depths of the FP32 3D semi-Lagrangian transport steps (Sec. 2.2): the number of z voxels each
 * thread of a 32 x 8 x depth brick interpolates from the brick's staged tile (4, 8 or 12), one for the
 * state steps and one for the adjoint steps. ga_setup picks each by timing its steps at every depth on
 * the context's own grid (state steps chained as in a sweep; cached per grid and model for the
 * process); every depth gives the same values bit for bit. ga_op_set_sl_depth overrides them (0
 * restores 8; GA_ERR_ARG for any value other than 0, 4, 8, 12). FP64 and 2D contexts keep 8 (their steps
 * are not tiled). CUDA graphs the context recorded earlier keep the depths they were recorded with. */
ga_status ga_op_get_sl_depth(const ga_ctx* ctx, int* state_depth, int* adjoint_depth);
ga_status ga_op_set_sl_depth(ga_ctx* ctx, int state_depth, int adjoint_depth);

/* Spectral divergence mu = sum_c d_c v_c. */
ga_status ga_op_div(ga_ctx* ctx, const void* v, void* mu);

/* Real-to-complex forward FFT of a scalar field over all dim axes, unnormalised, half spectrum
 * along the contiguous axis: fhat has n_1 x .. x (n_dim/2 + 1) complex entries (interleaved
 * re, im pairs of the element type), C order. ga_op_fft_c2r is the exact inverse (scaled by
 * 1/prod(n)) for Hermitian-consistent input. */
ga_status ga_op_fft_r2c(ga_ctx* ctx, const void* f, void* fhat);
ga_status ga_op_fft_c2r(ga_ctx* ctx, const void* fhat, void* f);

/* Lv = F^{-1}[|k|^{2s} F v] componentwise (s = reg_order); vector fields. */
ga_status ga_op_apply_L(ga_ctx* ctx, const void* v, void* Lv);

/* Leray projection P v = F^{-1}[(I - k~ k~^T/|k~|^2) F v] (Sec. 3.6); vector fields. */
ga_status ga_op_leray(ga_ctx* ctx, const void* v, void* pv);

/* FP64 compensated inner products out[i] = sum_j a[j] * b_i[j] over len elements of the
 * context element type, for i < count (count <= 64). b: device array of count device pointers
 * held in HOST memory (the pointer list itself is host memory); out: host memory. */
ga_status ga_op_dots(ga_ctx* ctx, const void* a, const void* const* b, int count, size_t len,
                     double* out);

/* NGMRES least squares on the device (Alg. 1, "arg min" line) from its FP64 Gram data:
 * beta = argmin || g_q + sum_i beta_i (g_q - g_i) ||_2, given c = <g_q, g_q>, a_i = <g_q, g_i>
 * and M_ij = <g_i, g_j> for i, j < m (m <= 63). Truncated symmetric eigen-solve of the normal
 * equations, dropping eigenvalues below 1e-14 * max. All arrays in HOST memory. */
ga_status ga_op_lsq(ga_ctx* ctx, int m, double c, const double* a, const double* M, double* beta);

/* Terminal state m(1) of the state equation for velocity v (the forward map of the
 * torch.autograd wrapper). v: vector field, m1_out: scalar field, in memory `mem`. */
ga_status ga_transport(ga_ctx* ctx, const void* v, void* m1_out, int mem);

/* Vector-Jacobian product of ga_transport in the optimise-then-discretise sense (Sec. 2.1):
 * for gamma = d loss / d m(1) (elementwise), grad_v = -b(lam1 = gamma) with b as in
 * ga_op_body_force. Elementwise (l2) gradients in and out. */
ga_status ga_transport_vjp(ga_ctx* ctx, const void* v, const void* gamma, void* grad_v, int mem);

/* Exact vector-Jacobian product of ga_transport (discretise-then-optimise): the gradient with respect
 * to the grid values of v of <gamma, m(1)(v)> for the discrete semi-Lagrangian transport (advection;
 * the incompressible model transports by advection too). GA_ERR_ARG for the continuity model.
 * Elementwise (l2) gradients in and out. */
ga_status ga_transport_vjp_exact(ga_ctx* ctx, const void* v, const void* gamma, void* grad_v, int mem);

/* Device-time accounting of one kernel class over a region of calls, with CUDA events recorded
 * on the context stream around every launch of that class: 0 = semi-Lagrangian state steps,
 * 1 = fused FFT-derivative passes of one field, 2 = 3D FFT transforms (all passes of one transform),
 * 3 = semi-Lagrangian adjoint steps, 4 = body-force derivative passes over two time steps. ga_prof_stop returns the summed event time (ms) and the
 * number of timed launches since ga_prof_start, and ends the accounting. */
ga_status ga_prof_start(ga_ctx* ctx, int kernel_class);
ga_status ga_prof_stop(ga_ctx* ctx, double* total_ms, long long* launches);

/* Number of CUDA kernels the library has launched in this process so far (all contexts). */
long long ga_kernel_launches(void);

/* Inner products for callers that cannot allocate device memory. The paper has no counterpart:
 * this is a convenience of the library. It computes the same FP64-accurate compensated inner
 * products as ga_op_dots, out[i] = sum_j a[j] * b_i[j] for i < count, without a context and without
 * calling cudaMalloc, cudaFree or any allocating routine. It is meant for programs that have handed
 * all device memory to their own allocator or pool, and for latency-critical loops that must not
 * pay for an allocation or the device-wide synchronisation that freeing implies.
 *   prec    GA_PREC_FP64 (a, b_i are double) or GA_PREC_MIXED (float); products are summed in FP64.
 *   a       device vector of len elements; b: HOST array of count device vectors of len elements.
 *   count   1..32: the per-CTA partial sums of all count products live in one fixed device array of
 *           32 * 608 doubles (155,648 bytes) defined in the library, which every GPU that loads the
 *           library holds until the process exits. count > 32 returns GA_ERR_ARG with a message.
 *   out     DEVICE array of count doubles, written in stream order.
 *   stream  cudaStream_t (NULL = legacy default stream); the call returns without synchronising.
 * The first call on a device looks up the device address of the fixed array (cudaGetSymbolAddress);
 * make that first call before any stream capture. The address is kept for the life of the process: a
 * device reset (cudaDeviceReset, or anything else that destroys the device's primary context) frees
 * the array, and the entry point must not be called on that device afterwards. Every call on a device shares the array and it
 * keeps the last call's contents (each call rewrites every partial it reads, so nothing needs
 * clearing); calls whose work overlaps on the GPU, e.g. on two streams at once, race on the array
 * and must be serialised by the caller. Errors: GA_ERR_ARG for null pointers, len 0, an unknown
 * precision or count outside 1..32; GA_ERR_CUDA for a launch failure; ga_last_error(NULL) holds the
 * reason. */
ga_status ga_dots_noalloc(int prec, const void* a, const void* const* b, int count, size_t len,
                          double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GA_OPS_H */
