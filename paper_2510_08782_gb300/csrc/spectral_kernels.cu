// Pointwise operators on the half spectrum (Sec. 2.2 diagonal scalings; Sec. 3.6 Leray projector).
//
// Half-spectrum entry (i0, i1, i2) has wavenumbers k_a = i_a for i_a <= n_a/2, else i_a - n_a
// (axis 2 stores only i2 <= n2/2). Even symbols use the full k (Nyquist included):
// L^ = |k|^{2s}. Derivative symbols use k~ (zero at the Nyquist index). The inverse (alpha L)^{-1}
// sets zero entries of L^ to one.
#include <cuda_runtime.h>

#include "kernels.h"

namespace ga {

namespace {

template <typename R> struct KVec {
  R k[3];   // full wavenumbers (even symbols)
  R kt[3];  // derivative wavenumbers
};

template <typename R> __device__ __forceinline__ KVec<R> kvec_of(const Grid& g, long long idx) {
  const int i2 = (int)(idx % g.n2h);
  const long long r = idx / g.n2h;
  const int i1 = (int)(r % g.n[1]);
  const int i0 = (int)(r / g.n[1]);
  const int ii[3] = {i0, i1, i2};
  KVec<R> kv;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int n = g.n[a];
    const int i = ii[a];
    const int k = (2 * i <= n) ? i : i - n;
    kv.k[a] = (R)k;
    kv.kt[a] = (2 * i == n) ? R(0) : (R)k;
  }
  return kv;
}

template <typename R> __device__ __forceinline__ R symbol_L(const KVec<R>& kv, int s) {
  const R k2 = kv.k[0] * kv.k[0] + kv.k[1] * kv.k[1] + kv.k[2] * kv.k[2];
  R r = k2;
  for (int i = 1; i < s; ++i) r *= k2;
  return r;
}

// Leray projection of the dim-component vector x (component c along axis 3 - dim + c).
template <typename T>
__device__ __forceinline__ void leray(const KVec<T>& kv, int dim, cx<T>* x) {
  T kc[3];
  T k2 = T(0);
  for (int c = 0; c < dim; ++c) {
    kc[c] = kv.kt[3 - dim + c];
    k2 += kc[c] * kc[c];
  }
  if (k2 == T(0)) return;
  T dr = T(0), di = T(0);
  for (int c = 0; c < dim; ++c) {
    dr += kc[c] * x[c].x;
    di += kc[c] * x[c].y;
  }
  dr /= k2;
  di /= k2;
  for (int c = 0; c < dim; ++c) {
    x[c].x -= kc[c] * dr;
    x[c].y -= kc[c] * di;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_spectral(Grid g, SpecArgs a, cx<T>* __restrict__ x) {
  const long long nh = g.nhalf;
  const int dim = g.dim;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nh;
       idx += (long long)gridDim.x * blockDim.x) {
    const KVec<T> kv = kvec_of<T>(g, idx);
    const T L = symbol_L<T>(kv, a.s);
    cx<T> xv[3];
    for (int c = 0; c < dim; ++c) xv[c] = x[c * nh + idx];
    if (a.mode == SPEC_APPLY_L || a.mode == SPEC_APPLY_ALPHA_L) {
      const T f = a.mode == SPEC_APPLY_L ? (T)L : (T)(a.alpha * L);
      for (int c = 0; c < dim; ++c) x[c * nh + idx] = cscale(xv[c], f);
      continue;
    }
    if (a.mode == SPEC_LERAY) {
      leray<T>(kv, dim, xv);
      for (int c = 0; c < dim; ++c) x[c * nh + idx] = xv[c];
      continue;
    }
    const T inv = T(-1) / ((T)a.alpha * (L == T(0) ? T(1) : L));
    if (a.mode == SPEC_PRECOND) {
      if (a.project) leray<T>(kv, dim, xv);
      for (int c = 0; c < dim; ++c) x[c * nh + idx] = cscale(xv[c], (T)inv);
      continue;
    }
  }
}

// t = alpha L s for s = -(alpha L)^{-1} g (Eq. (9)): alpha L^ s^ = -g^ wherever L^ != 0 and 0 at k = 0,
// so t_c = -(g_c - mean(g_c)), the mean read from the zero mode gh_c(0) = sum(g_c).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_neg_centered(const T* __restrict__ gv, const cx<T>* __restrict__ gh, T* __restrict__ t, long long nv, long long nh,
               int dim) {
  for (int c = 0; c < dim; ++c) {
    const T mean = gh[c * nh].x / (T)nv;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x)
      t[c * nv + i] = -(gv[c * nv + i] - mean);
  }
}

}  // namespace

template <typename T>
cudaError_t launch_spectral(const Grid& g, const SpecArgs& a, cx<T>* x, cudaStream_t st) {
  long long blocks = (g.nhalf + kThreads - 1) / kThreads;
  if (blocks > 152 * 8) blocks = 152 * 8;
  note_launches(1);
  k_spectral<T><<<(unsigned)blocks, kThreads, 0, st>>>(g, a, x);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_neg_centered(const Grid& g, const T* gv, const cx<T>* gh, T* t, cudaStream_t st) {
  long long blocks = (g.nvox + kThreads - 1) / kThreads;
  if (blocks > 152 * 8) blocks = 152 * 8;
  note_launches(1);
  k_neg_centered<T><<<(unsigned)blocks, kThreads, 0, st>>>(gv, gh, t, g.nvox, g.nhalf, g.dim);
  return cudaGetLastError();
}

template cudaError_t launch_spectral<float>(const Grid&, const SpecArgs&, cx<float>*, cudaStream_t);
template cudaError_t launch_spectral<double>(const Grid&, const SpecArgs&, cx<double>*, cudaStream_t);
template cudaError_t launch_neg_centered<float>(const Grid&, const float*, const cx<float>*, float*, cudaStream_t);
template cudaError_t launch_neg_centered<double>(const Grid&, const double*, const cx<double>*, double*, cudaStream_t);

}  // namespace ga
