// Semi-Lagrangian transport kernels (Sec. 2.2): RK2 departure points and one state / adjoint step.
//
// Interpolation is the periodic tensor-product cubic Lagrange interpolant on nodes {-1,0,1,2}
// (64 taps in 3D, 16 in 2D). Departure points are stored as displacements in grid units; the tap
// base index and the fraction are formed as i + floor(d) and d - floor(d), which is exact, so the
// fraction keeps full precision at any grid index. Indices wrap periodically for any displacement.
//
// Steps (stationary v, Heun characteristics; mu = div v):
//   state, advection   m_{j+1} = I[m_j](X-)
//   state, continuity  P = I[pi_j](X-), S = I[pi_j mu](X-), pi_{j+1} = P - h_t/2 (S + mu (P - h_t S))
//   adjoint, advection L = I[l_{j+1}](X+), S = I[l_{j+1} mu](X+), l_j = L + h_t/2 (S + mu (L + h_t S))
//   adjoint, continuity l_j = I[l_{j+1}](X+)
#include <cuda_runtime.h>

#include <type_traits>

#include "kernels.h"

namespace ga {

namespace {

template <typename T> struct Taps {
  int i[4];
  T w[4];
};

template <typename T> __device__ __forceinline__ T ga_floor(T x);
template <> __device__ __forceinline__ float ga_floor<float>(float x) { return floorf(x); }
template <> __device__ __forceinline__ double ga_floor<double>(double x) { return floor(x); }

// Taps of the cubic stencil for grid index `base` displaced by `disp` cells on an axis of n points.
template <typename T>
__device__ __forceinline__ void make_taps(int base, T disp, int n, Taps<T>& tp) {
  T fl = ga_floor<T>(disp);
  const T t = disp - fl;
  fl = fmin(fmax(fl, T(-1048576)), T(1048576));  // keeps the integer conversion defined for NaN/Inf
  int i0 = (base + (int)fl - 1) % n;
  if (i0 < 0) i0 += n;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    tp.i[k] = i0;
    i0 = (i0 + 1 == n) ? 0 : i0 + 1;
  }
  const T tp1 = t + T(1), tm1 = t - T(1), tm2 = t - T(2);
  const T sixth = T(1) / T(6);
  tp.w[0] = -t * tm1 * tm2 * sixth;
  tp.w[1] = tp1 * tm1 * tm2 * T(0.5);
  tp.w[2] = -tp1 * t * tm2 * T(0.5);
  tp.w[3] = tp1 * t * tm1 * sixth;
}

template <typename T> __device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// Interpolate f (and, with F2, the product f * g) at the stencil (tz, ty, tx).
template <typename T, int DIM, bool PROD>
__device__ __forceinline__ void gather(const T* __restrict__ f, const T* __restrict__ gfield,
                                       const Taps<T>& tz, const Taps<T>& ty, const Taps<T>& tx, int n1,
                                       int n2, T& out, T& outp) {
  T acc = T(0), accp = T(0);
#pragma unroll
  for (int a = 0; a < (DIM == 3 ? 4 : 1); ++a) {
    T ay = T(0), ayp = T(0);
    const size_t zoff = (DIM == 3) ? (size_t)tz.i[a] * n1 : 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const size_t roff = (zoff + ty.i[b]) * (size_t)n2;
      const T* row = f + roff;
      const T f0 = ldg(row + tx.i[0]), f1 = ldg(row + tx.i[1]), f2 = ldg(row + tx.i[2]),
              f3 = ldg(row + tx.i[3]);
      ay += ty.w[b] * (tx.w[0] * f0 + tx.w[1] * f1 + tx.w[2] * f2 + tx.w[3] * f3);
      if (PROD) {
        const T* grow = gfield + roff;
        ayp += ty.w[b] * (tx.w[0] * f0 * ldg(grow + tx.i[0]) + tx.w[1] * f1 * ldg(grow + tx.i[1]) +
                          tx.w[2] * f2 * ldg(grow + tx.i[2]) + tx.w[3] * f3 * ldg(grow + tx.i[3]));
      }
    }
    if (DIM == 3) {
      acc += tz.w[a] * ay;
      if (PROD) accp += tz.w[a] * ayp;
    } else {
      acc = ay;
      if (PROD) accp = ayp;
    }
  }
  out = acc;
  outp = accp;
}

struct Idx3 {
  int i0, i1, i2;
};
__device__ __forceinline__ Idx3 unflatten(long long idx, int n1, int n2) {
  Idx3 r;
  r.i2 = (int)(idx % n2);
  const long long q = idx / n2;
  r.i1 = (int)(q % n1);
  r.i0 = (int)(q / n1);
  return r;
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_departure(Grid g, const T* __restrict__ v, T* __restrict__ xm, T* __restrict__ xp, T ht) {
  const long long nv = g.nvox;
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const T h[3] = {T(6.283185307179586476925286766559) / T(n0), T(6.283185307179586476925286766559) / T(n1),
                  T(6.283185307179586476925286766559) / T(n2)};
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nv;
       idx += (long long)gridDim.x * blockDim.x) {
    const Idx3 p = unflatten(idx, n1, n2);
    T vc[3] = {T(0), T(0), T(0)};  // velocity along internal axes 0..2 (axis 0 unused in 2D)
#pragma unroll
    for (int c = 0; c < DIM; ++c) vc[3 - DIM + c] = v[c * nv + idx];
#pragma unroll
    for (int sgn = 0; sgn < 2; ++sgn) {
      const T sign = sgn == 0 ? T(1) : T(-1);  // +1: X- (state), -1: X+ (adjoint)
      Taps<T> tz, ty, tx;
      if (DIM == 3) make_taps<T>(p.i0, -sign * ht * vc[0] / h[0], n0, tz);
      make_taps<T>(p.i1, -sign * ht * vc[1] / h[1], n1, ty);
      make_taps<T>(p.i2, -sign * ht * vc[2] / h[2], n2, tx);
      T* out = sgn == 0 ? xm : xp;
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        const int ax = 3 - DIM + c;
        T vs, dummy;
        gather<T, DIM, false>(v + c * nv, nullptr, tz, ty, tx, n1, n2, vs, dummy);
        out[c * nv + idx] = -sign * T(0.5) * ht * (vc[ax] + vs) / h[ax];
      }
    }
  }
}

template <typename T, int DIM, int CONT>
__global__ void __launch_bounds__(kThreads)
k_sl_forward(Grid g, const T* __restrict__ m, const T* __restrict__ xm, const T* __restrict__ mu,
             T* __restrict__ out, T ht) {
  const long long nv = g.nvox;
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nv;
       idx += (long long)gridDim.x * blockDim.x) {
    const Idx3 p = unflatten(idx, n1, n2);
    Taps<T> tz, ty, tx;
    if (DIM == 3) make_taps<T>(p.i0, xm[idx], n0, tz);
    make_taps<T>(p.i1, xm[(DIM - 2) * nv + idx], n1, ty);
    make_taps<T>(p.i2, xm[(DIM - 1) * nv + idx], n2, tx);
    T P, S;
    gather<T, DIM, CONT != 0>(m, mu, tz, ty, tx, n1, n2, P, S);
    if (CONT) {
      const T mux = mu[idx];
      out[idx] = P - T(0.5) * ht * (S + mux * (P - ht * S));
    } else {
      out[idx] = P;
    }
  }
}

template <typename T, int DIM, int CONT>
__global__ void __launch_bounds__(kThreads)
k_sl_adjoint(Grid g, const T* __restrict__ lam, const T* __restrict__ xp, const T* __restrict__ mu,
             T* __restrict__ out, T ht) {
  const long long nv = g.nvox;
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nv;
       idx += (long long)gridDim.x * blockDim.x) {
    const Idx3 p = unflatten(idx, n1, n2);
    Taps<T> tz, ty, tx;
    if (DIM == 3) make_taps<T>(p.i0, xp[idx], n0, tz);
    make_taps<T>(p.i1, xp[(DIM - 2) * nv + idx], n1, ty);
    make_taps<T>(p.i2, xp[(DIM - 1) * nv + idx], n2, tx);
    T L, S;
    gather<T, DIM, CONT == 0>(lam, mu, tz, ty, tx, n1, n2, L, S);
    if (CONT) {
      out[idx] = L;
    } else {
      const T mux = mu[idx];
      out[idx] = L + T(0.5) * ht * (S + mux * (L + ht * S));
    }
  }
}

inline unsigned grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  const long long cap = 152LL * 16;
  return (unsigned)(b < cap ? b : cap);
}

}  // namespace

template <typename T>
cudaError_t launch_departure(const Grid& g, const T* v, T* xm, T* xp, T ht, cudaStream_t st, int both) {
  if constexpr (std::is_same<T, float>::value) {
    if (g.dim == 3) return launch_departure_tile(g, v, xm, xp, ht, both, st);
  }
  note_launches(1);
  if (g.dim == 3)
    k_departure<T, 3><<<grid_for(g.nvox), kThreads, 0, st>>>(g, v, xm, xp, ht);
  else
    k_departure<T, 2><<<grid_for(g.nvox), kThreads, 0, st>>>(g, v, xm, xp, ht);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sl_forward(const Grid& g, int continuity, const T* m, const T* xm, const T* mu, T* out,
                              T ht, cudaStream_t st, const cx<T>* qin, cx<T>* qout) {
  if constexpr (std::is_same<T, float>::value) {
    if (g.dim == 3) return launch_sl_tile(g, 0, continuity, m, xm, mu, out, ht, st, qin, qout);
  }
  const unsigned gr = grid_for(g.nvox);
  if (g.dim == 3) {
    if (continuity) {
      note_launches(1);
      k_sl_forward<T, 3, 1><<<gr, kThreads, 0, st>>>(g, m, xm, mu, out, ht);
    }
    else {
      note_launches(1);
      k_sl_forward<T, 3, 0><<<gr, kThreads, 0, st>>>(g, m, xm, mu, out, ht);
    }
  } else {
    if (continuity) {
      note_launches(1);
      k_sl_forward<T, 2, 1><<<gr, kThreads, 0, st>>>(g, m, xm, mu, out, ht);
    }
    else {
      note_launches(1);
      k_sl_forward<T, 2, 0><<<gr, kThreads, 0, st>>>(g, m, xm, mu, out, ht);
    }
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sl_adjoint(const Grid& g, int continuity, const T* lam, const T* xp, const T* mu, T* out,
                              T ht, cudaStream_t st, const cx<T>* qin, cx<T>* qout) {
  if constexpr (std::is_same<T, float>::value) {
    if (g.dim == 3) return launch_sl_tile(g, 1, continuity, lam, xp, mu, out, ht, st, qin, qout);
  }
  const unsigned gr = grid_for(g.nvox);
  if (g.dim == 3) {
    if (continuity) {
      note_launches(1);
      k_sl_adjoint<T, 3, 1><<<gr, kThreads, 0, st>>>(g, lam, xp, mu, out, ht);
    }
    else {
      note_launches(1);
      k_sl_adjoint<T, 3, 0><<<gr, kThreads, 0, st>>>(g, lam, xp, mu, out, ht);
    }
  } else {
    if (continuity) {
      note_launches(1);
      k_sl_adjoint<T, 2, 1><<<gr, kThreads, 0, st>>>(g, lam, xp, mu, out, ht);
    }
    else {
      note_launches(1);
      k_sl_adjoint<T, 2, 0><<<gr, kThreads, 0, st>>>(g, lam, xp, mu, out, ht);
    }
  }
  return cudaGetLastError();
}

#define GA_INST(T)                                                                                  \
  template cudaError_t launch_departure<T>(const Grid&, const T*, T*, T*, T, cudaStream_t, int);    \
  template cudaError_t launch_sl_forward<T>(const Grid&, int, const T*, const T*, const T*, T*, T,    \
                                            cudaStream_t, const cx<T>*, cx<T>*);                                           \
  template cudaError_t launch_sl_adjoint<T>(const Grid&, int, const T*, const T*, const T*, T*, T,    \
                                            cudaStream_t, const cx<T>*, cx<T>*);
GA_INST(float)
GA_INST(double)
#undef GA_INST

}  // namespace ga
