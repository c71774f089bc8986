// Control kernels of the device-driven solve: the scalar decisions of one iteration of Alg. 3 (or of
// RPGD) taken on the device, so that a whole solve is one CUDA graph whose conditional nodes loop
// over iterations and line-search trials and choose the kind of step.
//
// Each kernel runs as one thread and repeats, in the same FP64 operations and order, what the
// host-driven solver computes from the same device results:
//  * the Armijo test obj(v + rho s) < obj(v) + c rho <g, s> with the step halved on failure and the
//    accepted step remembered (doubled when the first trial was accepted), Eqs. (6)-(7), Sec. 2.3;
//  * the step kind of iteration k: a fixed-point (RPGD) step when mod(k, sigma + tau) >= sigma
//    (variant 1) or < tau (variant 2), Alg. 3; RPGD takes only fixed-point steps;
//  * the stop test ||g||_inf <= eps_rel ||g(v^(0))||_inf.
// Only these kernels set the conditional handles; each loop's condition turns false after a bounded
// number of passes (k reaches kmax; the line search stops after max_backtracks + 1 trials).
#include <cuda_runtime.h>

#include "kernels.h"

namespace ga {

namespace {

constexpr int kMethodRpgd = 1;  // ga_method value of RPGD

__device__ __forceinline__ bool one_thread() { return threadIdx.x == 0 && blockIdx.x == 0; }

__device__ __forceinline__ bool may_iterate(const ResCtl* c) {
  return c->started && c->status == 0 && c->k < c->kmax && !(c->stop_on_converged && c->converged);
}

__device__ __forceinline__ bool finite(double x) { return x == x && x - x == 0.0; }

__global__ void k_res_enter(ResCtl* c, cudaGraphConditionalHandle h_start) {
  if (one_thread()) cudaGraphSetConditional(h_start, c->started ? 0u : 1u);
}

__global__ void k_res_grad(ResCtl* c, const double* __restrict__ res, int which) {
  if (!one_thread()) return;
  const double m = 0.5 * c->hd * res[0];
  const double val = m + 0.5 * c->hd * res[1];
  const double ginf = res[2];
  c->grad_evals += 1;
  // a gradient at the accepted trial reuses the line search's state solve
  c->pde_solves += (which == RES_GRAD_ACCEPTED || which == RES_GRAD_TRIAL) ? 1 : 2;
  if (!finite(val) || !finite(ginf)) {
    if (c->status == 0) c->status = kResErrNan;
    return;
  }
  if (which == RES_GRAD_TRIAL) return;  // g(q) of an NGMRES step enters only the least squares
  c->ginf = ginf;
  if (which == RES_GRAD_START) {
    c->started = 1;
    c->k = 0;
    c->m = 0;
    c->head = c->W1 - 1;  // the first push fills slot 0
    c->J = val;
    c->mis = m;
    c->g0inf = ginf;
    c->rho_mem = 1.0;
    c->rel_grad_inf = ginf > 0.0 ? 1.0 : 0.0;
    c->converged = c->rel_grad_inf <= c->rel_tol ? 1 : 0;
  } else {
    c->Jn = val;
    c->misn = m;
  }
}

__global__ void k_res_pushed(ResCtl* c, int iteration, cudaGraphConditionalHandle h_iter) {
  if (!one_thread()) return;
  if (c->status == 0) {
    c->head = (c->head + 1) % c->W1;
    c->m = c->m + 1 < c->W1 ? c->m + 1 : c->W1;
    if (iteration) {
      c->k += 1;
      c->J = c->Jn;
      c->mis = c->misn;
      c->last_branch = c->branch == 0 ? 1 : 0;
      c->fp_steps += c->branch == 0 ? 1 : 0;
      c->rel_grad_inf = c->g0inf > 0.0 ? c->ginf / c->g0inf : 0.0;
      c->converged = c->rel_grad_inf <= c->rel_tol ? 1 : 0;
    }
  }
  if (iteration) cudaGraphSetConditional(h_iter, may_iterate(c) ? 1u : 0u);
}

__global__ void k_res_loop_cond(ResCtl* c, cudaGraphConditionalHandle h_iter) {
  if (one_thread()) cudaGraphSetConditional(h_iter, may_iterate(c) ? 1u : 0u);
}

__global__ void k_res_ls_begin(ResCtl* c, const double* __restrict__ gs_raw, cudaGraphConditionalHandle h_ls) {
  if (!one_thread()) return;
  c->gs = c->hd * gs_raw[0];
  c->rho = c->rho_mem;
  c->trial = 0;
  cudaGraphSetConditional(h_ls, c->status == 0 ? 1u : 0u);
}

__global__ void k_res_ls_check(ResCtl* c, const double* __restrict__ res, cudaGraphConditionalHandle h_ls) {
  if (!one_thread()) return;
  const double m = 0.5 * c->hd * res[0];
  const double jq = m + 0.5 * c->hd * res[1];
  c->trial += 1;
  c->ls_trials += 1;
  c->obj_evals += 1;
  c->pde_solves += 1;
  unsigned more = 0u;
  if (jq < c->J + c->armijo_c * c->rho * c->gs) {
    c->rho_mem = c->trial == 1 ? 2.0 * c->rho : c->rho;
    c->last_rho = c->rho;
  } else {
    c->rho *= 0.5;
    if (c->trial > c->max_backtracks) c->status = kResErrLinesearch;
    else more = 1u;
  }
  cudaGraphSetConditional(h_ls, more);
}

__global__ void k_res_branch(ResCtl* c, cudaGraphConditionalHandle h_sw) {
  if (!one_thread()) return;
  int b = 2;
  if (c->status == 0) {
    const int per = c->sigma + c->tau;
    const int r = per > 0 ? c->k % per : 0;
    const bool fp = c->method == kMethodRpgd || (c->variant == 2 ? r < c->tau : r >= c->sigma);
    b = fp ? 0 : 1;
  }
  c->branch = b;
  cudaGraphSetConditional(h_sw, (unsigned)b);
}

}  // namespace

cudaError_t launch_res_enter(ResCtl* c, cudaGraphConditionalHandle h_start, cudaStream_t st) {
  note_launches(1);
  k_res_enter<<<1, 32, 0, st>>>(c, h_start);
  return cudaGetLastError();
}
cudaError_t launch_res_grad(ResCtl* c, const double* res, int which, cudaStream_t st) {
  note_launches(1);
  k_res_grad<<<1, 32, 0, st>>>(c, res, which);
  return cudaGetLastError();
}
cudaError_t launch_res_pushed(ResCtl* c, int iteration, cudaGraphConditionalHandle h_iter, cudaStream_t st) {
  note_launches(1);
  k_res_pushed<<<1, 32, 0, st>>>(c, iteration, h_iter);
  return cudaGetLastError();
}
cudaError_t launch_res_loop_cond(ResCtl* c, cudaGraphConditionalHandle h_iter, cudaStream_t st) {
  note_launches(1);
  k_res_loop_cond<<<1, 32, 0, st>>>(c, h_iter);
  return cudaGetLastError();
}
cudaError_t launch_res_ls_begin(ResCtl* c, const double* gs_raw, cudaGraphConditionalHandle h_ls, cudaStream_t st) {
  note_launches(1);
  k_res_ls_begin<<<1, 32, 0, st>>>(c, gs_raw, h_ls);
  return cudaGetLastError();
}
cudaError_t launch_res_ls_check(ResCtl* c, const double* res, cudaGraphConditionalHandle h_ls, cudaStream_t st) {
  note_launches(1);
  k_res_ls_check<<<1, 32, 0, st>>>(c, res, h_ls);
  return cudaGetLastError();
}
cudaError_t launch_res_branch(ResCtl* c, cudaGraphConditionalHandle h_sw, cudaStream_t st) {
  note_launches(1);
  k_res_branch<<<1, 32, 0, st>>>(c, h_sw);
  return cudaGetLastError();
}

}  // namespace ga
