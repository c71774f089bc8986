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
k_spectral(Grid g, SpecArgs a, cx<T>* __restrict__ x, cx<T>* __restrict__ v) {
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
    // SPEC_EPILOGUE: g^ = alpha L^ v^ + (P) b^ ; optionally s^ = -(P g^) / (alpha L^_fix)
    if (a.project) leray<T>(kv, dim, xv);
    cx<T> gv[3];
    const T aL = (T)(a.alpha * L);
    for (int c = 0; c < dim; ++c) {
      const cx<T> vv = v[c * nh + idx];
      gv[c] = mk<T>(aL * vv.x + xv[c].x, aL * vv.y + xv[c].y);
      x[c * nh + idx] = gv[c];
    }
    if (a.want_s) {
      if (a.project) leray<T>(kv, dim, gv);
      for (int c = 0; c < dim; ++c) v[c * nh + idx] = cscale(gv[c], (T)inv);
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

// sum over the half spectrum of w(k) |k|^{2s} |v^_c(k)|^2 (w = 1 on the k2 = 0 and Nyquist planes,
// 2 elsewhere). Terms are formed in the element type; each thread accumulates them in a compensated
// (double-float for FP32) sum, CTAs combine in FP64.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_reg_sum(Grid g, int s, const cx<T>* __restrict__ vh, double* __restrict__ partial) {
  const long long nh = g.nhalf;
  T hi = T(0), lo = T(0);
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nh;
       idx += (long long)gridDim.x * blockDim.x) {
    const KVec<T> kv = kvec_of<T>(g, idx);
    const int i2 = (int)(idx % g.n2h);
    const T w = (i2 == 0 || 2 * i2 == g.n[2]) ? T(1) : T(2);
    T e = T(0);
    for (int c = 0; c < g.dim; ++c) {
      const cx<T> z = vh[c * nh + idx];
      e += z.x * z.x + z.y * z.y;
    }
    const T term = w * symbol_L<T>(kv, s) * e;
    const T t = hi + term;  // two-sum
    const T bb = t - hi;
    lo += (hi - (t - bb)) + (term - bb);
    hi = t;
  }
  double acc = (double)hi + (double)lo;
  __shared__ double red[kThreads / 32];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double r = threadIdx.x < kThreads / 32 ? red[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) r += __shfl_down_sync(0xffffffffu, r, off);
    if (threadIdx.x == 0) partial[blockIdx.x] = r;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_spectral(const Grid& g, const SpecArgs& a, cx<T>* x, cx<T>* v, cudaStream_t st) {
  long long blocks = (g.nhalf + kThreads - 1) / kThreads;
  if (blocks > 152 * 8) blocks = 152 * 8;
  note_launches(1);
  k_spectral<T><<<(unsigned)blocks, kThreads, 0, st>>>(g, a, x, v);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_reg_sum(const Grid& g, int s, const cx<T>* vh, double* partial, cudaStream_t st) {
  note_launches(1);
  k_reg_sum<T><<<kRedBlocks, kThreads, 0, st>>>(g, s, vh, partial);
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

template cudaError_t launch_spectral<float>(const Grid&, const SpecArgs&, cx<float>*, cx<float>*, cudaStream_t);
template cudaError_t launch_spectral<double>(const Grid&, const SpecArgs&, cx<double>*, cx<double>*, cudaStream_t);
template cudaError_t launch_reg_sum<float>(const Grid&, int, const cx<float>*, double*, cudaStream_t);
template cudaError_t launch_reg_sum<double>(const Grid&, int, const cx<double>*, double*, cudaStream_t);
template cudaError_t launch_neg_centered<float>(const Grid&, const float*, const cx<float>*, float*, cudaStream_t);
template cudaError_t launch_neg_centered<double>(const Grid&, const double*, const cx<double>*, double*, cudaStream_t);

}  // namespace ga
